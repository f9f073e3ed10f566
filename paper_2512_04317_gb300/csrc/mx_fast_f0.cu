// Register-resident MX pass instantiated for the E4M3 element format.
#include "mx_fast_kernel.cuh"

namespace mxfft {
namespace fast {
template cudaError_t launch_fast_fmt<0>(const FastArgs&, int, int, cudaStream_t);
}  // namespace fast
MX_BOUNDS_COUNTER(fast_f0)
}  // namespace mxfft
