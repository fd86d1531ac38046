// Double-precision instances of the FFT pipeline kernels.
#include "fft_kernels.inc"

namespace wgw {

WGW_INST_FFT(double, double)

}  // namespace wgw
