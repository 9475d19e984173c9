// Kernel family: row pass, double, d = 2.
#include "lsfft_dispatch.cuh"
namespace lsfft {
LSFFT_DEFINE_ROW_DISPATCH(double, 2)
}  // namespace lsfft
