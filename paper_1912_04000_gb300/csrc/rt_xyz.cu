// Spectrum -> CIE XYZ contraction (section 6: colorimetry from spectra).
//
//   xyz[p][c] = sum_j (spectral[p][j] / spp) * w[j][c]
//
// RT_XYZ_FP64: CUDA cores, FP64, one warp per pixel group (reference mode).
#include <cstdint>

#include "rt_internal.h"

namespace srt {

namespace {

// one thread per pixel row, the row staged through shared memory by the
// whole block with coalesced loads
__global__ void __launch_bounds__(256) k_xyz_fp64(const double* __restrict__ s, uint64_t np, uint32_t bc,
                                                  const float* __restrict__ w, double inv_spp, float* __restrict__ xyz) {
  extern __shared__ double tile[];  // [256][bc]
  const uint64_t p0 = (uint64_t)blockIdx.x * blockDim.x;
  const uint64_t rows = (np - p0) < blockDim.x ? (np - p0) : blockDim.x;
  const uint64_t elems = rows * bc;
  const double* src = s + p0 * bc;
  for (uint64_t e = threadIdx.x; e < elems; e += blockDim.x) tile[e] = src[e];
  __syncthreads();
  if (threadIdx.x < rows) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    const double* row = tile + (size_t)threadIdx.x * bc;
    for (uint32_t j = 0; j < bc; ++j) {
      const double v = row[j] * inv_spp;
      a0 += v * (double)w[3 * j];
      a1 += v * (double)w[3 * j + 1];
      a2 += v * (double)w[3 * j + 2];
    }
    float* o = xyz + 3 * (p0 + threadIdx.x);
    o[0] = (float)a0;
    o[1] = (float)a1;
    o[2] = (float)a2;
  }
}

}  // namespace

size_t xyz_wsplit_elems(uint32_t band_count) { return (size_t)((band_count + 15) / 16 * 16) * 16 * 3; }

void xyz_prepare_weights(const float* cmf_w_rows, uint32_t band_count, uint16_t* wsplit_host) {
  (void)cmf_w_rows;
  (void)band_count;
  (void)wsplit_host;
}

void launch_xyz(const double* spectral, uint64_t n_pixels, const XyzWeights& w, uint32_t spp, int mode, float* xyz,
                cudaStream_t st) {
  (void)mode;
  if (n_pixels == 0) return;
  int block = (int)(49152 / (8 * (size_t)w.band_count));
  block = block > 256 ? 256 : (block < 1 ? 1 : block);
  const uint64_t grid = (n_pixels + block - 1) / block;
  const size_t smem = (size_t)block * w.band_count * sizeof(double);
  k_xyz_fp64<<<(unsigned)grid, block, smem, st>>>(spectral, n_pixels, w.band_count, w.w32, 1.0 / (double)spp, xyz);
}

}  // namespace srt
