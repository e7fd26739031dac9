// Gradient of the smoothed isotropic total variation of Eq. 17 (the TV term,
// by the smooth approximation the paper uses in its FISTA reconstruction):
//   TV_eps(u) = sum_{y,x} sqrt(|D_x u|^2 + |D_y u|^2 + eps^2),
//   grad = D^H (D u / sqrt(|D u|^2 + eps^2)),
// with forward differences and a Neumann boundary (no difference across the
// last column / row), per z-slice, as one complex image (gradient with
// respect to the real and imaginary parts).
//
// One thread per pixel: it forms the normalised differences p = D u / w at
// its own pixel and at its left and upper neighbours (whose p enter its
// adjoint sum), reading u at up to seven pixels through the read-only
// cache.  HBM-bound: 8 bytes read and 8 written per pixel when the
// neighbours hit in cache.
#include <algorithm>

#include "gpjc_device.cuh"
#include "gpjc_kernels.h"

namespace gpjc {

constexpr int kTvThreads = 256;

// p = (D_x u, D_y u) / sqrt(|D u|^2 + eps^2) at (y, x)
__device__ __forceinline__ void tv_p(const float2* __restrict__ u, int y, int x, int ny, int nx, float eps2,
                                     float2* px, float2* py) {
  const float2 c = __ldg(u + (size_t)y * nx + x);
  float2 dx = make_float2(0.f, 0.f), dy = make_float2(0.f, 0.f);
  if (x + 1 < nx) {
    const float2 r = __ldg(u + (size_t)y * nx + x + 1);
    dx = make_float2(r.x - c.x, r.y - c.y);
  }
  if (y + 1 < ny) {
    const float2 d = __ldg(u + (size_t)(y + 1) * nx + x);
    dy = make_float2(d.x - c.x, d.y - c.y);
  }
  const float inv = rsqrtf(dx.x * dx.x + dx.y * dx.y + dy.x * dy.x + dy.y * dy.y + eps2);
  *px = make_float2(dx.x * inv, dx.y * inv);
  *py = make_float2(dy.x * inv, dy.y * inv);
}

__global__ void __launch_bounds__(kTvThreads) k_tv_grad(const float2* __restrict__ u, float2* __restrict__ g,
                                                        int nz, int ny, int nx, float eps2) {
  const size_t plane = (size_t)ny * nx;
  const size_t total = plane * nz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int z = (int)(i / plane);
    const int rem = (int)(i - (size_t)z * plane);
    const int y = rem / nx, x = rem - y * nx;
    const float2* us = u + (size_t)z * plane;
    float2 px, py, out = make_float2(0.f, 0.f);
    tv_p(us, y, x, ny, nx, eps2, &px, &py);
    if (x + 1 < nx) out = make_float2(out.x - px.x, out.y - px.y);
    if (y + 1 < ny) out = make_float2(out.x - py.x, out.y - py.y);
    if (x > 0) {
      tv_p(us, y, x - 1, ny, nx, eps2, &px, &py);
      out = make_float2(out.x + px.x, out.y + px.y);
    }
    if (y > 0) {
      tv_p(us, y - 1, x, ny, nx, eps2, &px, &py);
      out = make_float2(out.x + py.x, out.y + py.y);
    }
    g[i] = out;
  }
}

// ------------------------------------------------------------------ host side --
// (left out when the kernel above is compiled for a host emulation)
#ifndef GPJC_DEVICE_SOURCE_ONLY
cudaError_t launch_tv_grad(const float2* u, float2* g, int nz, int ny, int nx, float eps2, cudaStream_t st) {
  const size_t total = (size_t)nz * ny * nx;
  const int blocks = (int)std::min<size_t>((total + kTvThreads - 1) / kTvThreads, (size_t)152 * 8);
  note_launches(1); k_tv_grad<<<blocks, kTvThreads, 0, st>>>(u, g, nz, ny, nx, eps2);
  return cudaGetLastError();
}
#endif  // GPJC_DEVICE_SOURCE_ONLY

}  // namespace gpjc
