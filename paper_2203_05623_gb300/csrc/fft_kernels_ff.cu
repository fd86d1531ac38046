// Instances of the FFT pipeline kernels that read and write FP64 arrays and compute in
// float-float arithmetic (pair intermediates and twiddles in float-float as well).
#include "fft_kernels.inc"

namespace wgw {

WGW_INST_FFT(double, ff)

}  // namespace wgw
