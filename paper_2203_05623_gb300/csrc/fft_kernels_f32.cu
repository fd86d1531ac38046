// Single-precision instances of the FFT pipeline kernels.
#include "fft_kernels.inc"

namespace wgw {

// Threads of the shared-memory FFT kernels.  At N >= 96 one CTA fills most of an SM's shared memory
// (a float-float 96 x 97 plane is 149 KB), so 512 threads keep 16 warps per SM instead of 8.
int fft_threads(int n) { return n >= 96 ? 512 : (n >= 40 ? 256 : 128); }

WGW_INST_FFT(float, float)

}  // namespace wgw
