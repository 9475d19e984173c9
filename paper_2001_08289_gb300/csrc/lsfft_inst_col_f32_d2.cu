// Kernel family: col pass, float, d = 2.
#include "lsfft_dispatch.cuh"
namespace lsfft {
LSFFT_DEFINE_COL_DISPATCH(float, 2)
}  // namespace lsfft
