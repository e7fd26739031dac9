// Readout stage of E_c^H, FP32 register-tiled kernel with tiles of 2
// readout samples (Eq. 15, adjoint; patch widths that are not multiples of 4).
#include "k_readout.cuh"

namespace gpjc {

template <int MAXX, int TS>
static cudaError_t launch_a(const Geo& g, const RTiles& tl, const float2* H2, const float2* coil,
                            const float2* A, float2* xpart, int nchunk, cudaStream_t st) {
  const int cpc = (g.nc + nchunk - 1) / nchunk;
  const size_t sm = readout_adj_smem(g, tl.rb, tl.hstage);
  static int attr = 0;
  if ((int)sm > attr) {
    cudaFuncSetAttribute(k1a_tiled<MAXX, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k1a_tiled<MAXX, TS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         readout_carveout((const void*)k1a_tiled<MAXX, TS>, sm));
    attr = (int)sm;
  }
  dim3 grid((g.rows + tl.rb - 1) / tl.rb, nchunk);
  note_launches(1); k1a_tiled<MAXX, TS><<<grid, kRThreads, sm, st>>>(g, tl, H2, coil, A, xpart, cpc);
  return cudaGetLastError();
}

cudaError_t launch_k1a_tiled_ts2(const Geo& g, const RTiles& tl, const float2* H2, const float2* coil,
                                 const float2* A, float2* xpart, int nchunk, cudaStream_t st) {
  const int mx = (tl.rb * g.nx + kRThreads - 1) / kRThreads;
  if (mx <= 1) return launch_a<1, 2>(g, tl, H2, coil, A, xpart, nchunk, st);
  if (mx <= 2) return launch_a<2, 2>(g, tl, H2, coil, A, xpart, nchunk, st);
  return cudaErrorInvalidValue;
}

}  // namespace gpjc
