// Kernel family: row pass, float, d = 2.
#include "lsfft_dispatch.cuh"
namespace lsfft {
LSFFT_DEFINE_ROW_DISPATCH(float, 2)
}  // namespace lsfft
