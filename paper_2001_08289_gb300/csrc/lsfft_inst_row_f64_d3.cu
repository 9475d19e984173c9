// Kernel family: row pass, double, d = 3.
#include "lsfft_dispatch.cuh"
namespace lsfft {
LSFFT_DEFINE_ROW_DISPATCH(double, 3)
}  // namespace lsfft
