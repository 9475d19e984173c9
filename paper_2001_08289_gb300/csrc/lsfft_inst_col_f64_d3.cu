// Kernel family: col pass, double, d = 3.
#include "lsfft_dispatch.cuh"
namespace lsfft {
LSFFT_DEFINE_COL_DISPATCH(double, 3)
}  // namespace lsfft
