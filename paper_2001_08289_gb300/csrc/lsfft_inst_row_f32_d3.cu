// Kernel family: row pass, float, d = 3.
#include "lsfft_dispatch.cuh"
namespace lsfft {
LSFFT_DEFINE_ROW_DISPATCH(float, 3)
}  // namespace lsfft
