// Instantiations of the fused x pass (qw_spectral_dev.cuh) for one group of line
// lengths; the groups live in separate units so that they compile in parallel.
#include "qw_spectral_dev.cuh"

namespace qw {
QW_FUSED_LENGTHS_2(QW_FUSED_X_INSTANTIATE)
}  // namespace qw
