// Single-precision instances of the FFT pipeline kernels.
#include "fft_kernels.inc"

namespace wgw {

int fft_threads(int n) { return n >= 40 ? 256 : 128; }

WGW_INST_FFT(float, float)

}  // namespace wgw
