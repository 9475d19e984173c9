// Kernel family: col pass, float, d = 3.
#include "lsfft_dispatch.cuh"
namespace lsfft {
LSFFT_DEFINE_COL_DISPATCH(float, 3)
}  // namespace lsfft
