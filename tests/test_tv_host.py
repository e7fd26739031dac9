"""The smoothed-TV gradient kernel (csrc/k_tv.cu), compiled for the host
with g++ and run over its whole grid (one emulated thread at a time: the
kernel has no barriers), against the oracle's gradient of Eq. 17's TV term
on a ragged 3-slice image.  This pins the device source's stencil and
boundary handling independently of a GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2601_05418_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2601_05418_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

DRIVER = r"""
#include <cuda_runtime.h>
#include <cmath>
#include <cstdio>
#include <vector>
template <class T> static inline T __ldg(const T* p) { return *p; }
template <class T> static inline T __ldcg(const T* p) { return *p; }
template <class T> static inline T __shfl_xor_sync(unsigned, T v, int) { return v; }
static inline void __syncthreads() {}
static inline void __threadfence() {}
static inline float rsqrtf(float v) { return 1.0f / std::sqrt(v); }
#define sincospif(a, s, c) (*(s) = std::sin(M_PI * (a)), *(c) = std::cos(M_PI * (a)))
static inline double atomicAdd(double* p, double v) { double o = *p; *p += v; return o; }
static inline unsigned atomicAdd(unsigned* p, unsigned v) { unsigned o = *p; *p += v; return o; }
template <class T> static inline T atomicInc(T* p, T) { return (*p)++; }
static uint3 threadIdx, blockIdx;
static dim3 blockDim, gridDim;
#undef __global__
#define __global__
#undef __launch_bounds__
#define __launch_bounds__(...)
#define GPJC_DEVICE_SOURCE_ONLY
#include "k_tv.cu"
using namespace gpjc;

int main() {
  int nz, ny, nx;
  double eps;
  if (scanf("%d %d %d %lf", &nz, &ny, &nx, &eps) != 4) return 2;
  const size_t n = (size_t)nz * ny * nx;
  std::vector<float2> u(n), g(n);
  for (auto& v : u) if (scanf("%f %f", &v.x, &v.y) != 2) return 3;
  blockDim = dim3(256, 1, 1);
  gridDim = dim3(3, 1, 1);  // fewer threads than pixels: the grid-stride loop runs
  for (unsigned b = 0; b < gridDim.x; ++b)
    for (unsigned t = 0; t < blockDim.x; ++t) {
      blockIdx = make_uint3(b, 0, 0);
      threadIdx = make_uint3(t, 0, 0);
      k_tv_grad(u.data(), g.data(), nz, ny, nx, (float)(eps * eps));
    }
  for (auto& v : g) printf("%.9e %.9e\n", v.x, v.y);
  return 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None or not os.path.isdir(CUDA_INC), reason="needs g++ and CUDA headers")
def test_tv_gradient_kernel_matches_oracle(tmp_path):
    nz, ny, nx, eps = 3, 13, 19, 0.05
    src = tmp_path / "tv_driver.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "tv_driver"
    r = subprocess.run(["g++", "-O1", "-std=c++17", "-w", "-I", CUDA_INC, "-I", CSRC, "-x", "c++", str(src),
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    u = synth.complex_normal((nz, ny, nx), 111)
    u[1] = 0.3  # a constant slice: zero gradient
    inp = f"{nz} {ny} {nx} {eps}\n" + "\n".join(f"{v.real:.9e} {v.imag:.9e}" for v in u.ravel())
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr[-2000:]
    vals = np.array(out.stdout.split(), np.float64).reshape(-1, 2)
    g = (vals[:, 0] + 1j * vals[:, 1]).reshape(nz, ny, nx)
    ref = np.stack([O.tv_smooth_grad(u[k], eps) for k in range(nz)])
    assert np.linalg.norm(g - ref) < 1e-5 * np.linalg.norm(ref)
    assert np.abs(g[1]).max() == 0.0
