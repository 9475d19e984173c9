// Kernel family: col pass, double, d = 2.
#include "lsfft_dispatch.cuh"
namespace lsfft {
LSFFT_DEFINE_COL_DISPATCH(double, 2)
}  // namespace lsfft
