"""The readout-model kernels of the 16-bit operators (two coils per FFT
call), compiled for the host with g++ and run as 256 emulated threads per
block (std::thread, with a real barrier for __syncthreads), against the
oracle's readout stage: V[row][n][t] = e^{-i phi(t,y)} DFT_x{pad(c_n rho)}(t)
and its adjoint.  Odd coil count and two coil chunks, so both the two-coil
and the one-coil pass run.  This pins the index arithmetic of the device
source itself, independently of a GPU."""
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
#include <barrier>
#include <cmath>
#include <cstdio>
#include <functional>
#include <thread>
#include <vector>
static std::barrier<>* g_bar = nullptr;
static inline void __syncthreads() { g_bar->arrive_and_wait(); }
template <class T> static inline T __ldg(const T* p) { return *p; }
template <class T> static inline T __ldcg(const T* p) { return *p; }
template <class T> static inline T __shfl_xor_sync(unsigned, T v, int) { return v; }
static inline void __threadfence() {}
#define sincospif(a, s, c) (*(s) = std::sin(M_PI * (a)), *(c) = std::cos(M_PI * (a)))
static inline double atomicAdd(double* p, double v) { double o = *p; *p += v; return o; }
static inline unsigned atomicAdd(unsigned* p, unsigned v) { unsigned o = *p; *p += v; return o; }
template <class T> static inline T atomicInc(T* p, T) { return (*p)++; }
static inline int min(int a, int b) { return a < b ? a : b; }
static thread_local uint3 threadIdx;
static uint3 blockIdx;
static dim3 blockDim, gridDim;
#undef __global__
#define __global__
#undef __shared__
#define __shared__
#undef __launch_bounds__
#define __launch_bounds__(...)
#define GPJC_DEVICE_SOURCE_ONLY
#include "k_sim.cu"
namespace gpjc {
float2 smem[1 << 16];
}
using namespace gpjc;

static void plan(int n, FftPlan* pl) {
  pl->n = n; pl->nst = 0; pl->n1 = pl->n2 = 0;
  int m = n;
  for (int R : {8, 4, 2, 7, 5, 3}) while (m % R == 0) { pl->rad[pl->nst++] = R; m /= R; }
  for (int n1 : {16, 8}) if (n % n1 == 0 && fft2p_supported(n1, n / n1)) { pl->n1 = n1; pl->n2 = n / n1; break; }
}

// one block of 256 emulated threads
static void run_block(int bx, int by, const std::function<void()>& body) {
  blockIdx = make_uint3(bx, by, 0);
  std::barrier<> bar(256);
  g_bar = &bar;
  std::vector<std::thread> th;
  for (int t = 0; t < 256; ++t)
    th.emplace_back([t, &body] { threadIdx = make_uint3(t, 0, 0); body(); });
  for (auto& x : th) x.join();
}

int main() {
  int nx, ny, nc, os, nchunk;
  double cycles, kappa;
  if (scanf("%d %d %d %d %d %lf %lf", &nx, &ny, &nc, &os, &nchunk, &cycles, &kappa) != 7) return 2;
  const int ntx = os * nx, rows = ny;
  Geo g = {};
  g.nx = nx; g.ny = ny; g.nz = 1; g.nc = nc; g.os = os; g.ntx = ntx; g.rows = rows;
  plan(nx, &g.fx);
  if (!g.fx.n1) return 3;
  std::vector<float2> tw(nx), pre(os * nx), post(ny * ntx), postz(ntx, make_float2(1.f, 0.f));
  for (int k = 0; k < nx; ++k) {
    const int e = (k % g.fx.n2) * (k / g.fx.n2);
    tw[k] = make_float2((float)std::cos(-2 * M_PI * e / nx), (float)std::sin(-2 * M_PI * e / nx));
  }
  for (int s = 0; s < os; ++s)
    for (int x = 0; x < nx; ++x) {
      const double a = -2 * M_PI * (double)((s * x) % ntx) / ntx, sg = (x & 1) ? -1.0 : 1.0;
      pre[s * nx + x] = make_float2((float)(sg * std::cos(a)), (float)(sg * std::sin(a)));
    }
  for (int y = 0; y < ny; ++y)
    for (int t = 0; t < ntx; ++t) {
      const int m = t / os, s = t - m * os;
      const double ay = kappa * (1 - std::cos(2 * M_PI * cycles * t / ntx)) / 2;
      const double a = M_PI * s / os - 2 * M_PI * ay * (y - ny / 2) / ny;
      const double sc = (((m + nx / 2) & 1) ? -1.0 : 1.0) / std::sqrt((double)ntx);
      post[y * ntx + t] = make_float2((float)(sc * std::cos(a)), (float)(sc * std::sin(a)));
    }
  g.tw_x = tw.data(); g.pre = pre.data(); g.post_y = post.data(); g.post_z = postz.data();
  const size_t L = (size_t)rows * nx;
  std::vector<float2> x(L), coil(nc * L), V((size_t)rows * nc * ntx), W((size_t)rows * nc * ntx),
      xpart((size_t)nchunk * L);
  for (auto& v : x) if (scanf("%f %f", &v.x, &v.y) != 2) return 4;
  for (auto& v : coil) if (scanf("%f %f", &v.x, &v.y) != 2) return 4;
  for (auto& v : W) if (scanf("%f %f", &v.x, &v.y) != 2) return 4;
  blockDim = dim3(256, 1, 1);
  const int cpc = (nc + nchunk - 1) / nchunk;
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < nchunk; ++c) {
      run_block(r, c, [&] { k1_sim_fwd2<float2, 2>(g, x.data(), coil.data(), V.data(), cpc, 0); });
      if (nx <= 256)  // one output pixel per thread, as the library launches it
        run_block(r, c, [&] { k1_sim_adj2<float2, 2, 1>(g, W.data(), coil.data(), xpart.data(), cpc, 0); });
      else
        run_block(r, c, [&] { k1_sim_adj2<float2, 2, 2>(g, W.data(), coil.data(), xpart.data(), cpc, 0); });
    }
  for (auto& v : V) printf("%.9e %.9e\n", v.x, v.y);
  for (size_t i = 0; i < L; ++i) {
    float2 s = make_float2(0.f, 0.f);
    for (int c = 0; c < nchunk; ++c) { s.x += xpart[c * L + i].x; s.y += xpart[c * L + i].y; }
    printf("%.9e %.9e\n", s.x, s.y);
  }
  return 0;
}
"""


def _flat(a):
    a = np.asarray(a, np.complex128).ravel()
    return "\n".join(f"{v.real:.9e} {v.imag:.9e}" for v in a)


@pytest.mark.skipif(shutil.which("g++") is None or not os.path.isdir(CUDA_INC), reason="needs g++ and CUDA headers")
@pytest.mark.parametrize("nx,ny,os_", [(40, 6, 2), (320, 2, 8)])
def test_two_coil_readout_model_kernels_match_oracle(tmp_path, nx, ny, os_):
    """40 points (8 x 5) at 2x, one output pixel per thread; 320 points
    (16 x 20) at 8x: 16 transforms of 20 rows exceed the 256 threads (two
    tasks per thread in the FFT passes) and the adjoint keeps two output
    pixels per thread."""
    nc, nchunk, cycles, kappa = 3, 2, 2.0, 1.3
    src = tmp_path / "sim_driver.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "sim_driver"
    r = subprocess.run(["g++", "-O1", "-std=c++20", "-pthread", "-w", "-I", CUDA_INC, "-I", CSRC, "-x", "c++",
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    g = synth.tiny_geometry(nx=nx, ny=ny, nc=nc, os=os_, cycles=cycles, kappa_y=kappa, n_groups=2)
    coils = synth.coil_maps(nx, ny, 1, nc, 71)
    x = synth.complex_normal(g.shape, 72)
    W = synth.complex_normal((ny, nc, g.ntx), 73)  # spectra [row][coil][t]
    inp = f"{nx} {ny} {nc} {os_} {nchunk} {cycles} {kappa}\n" + "\n".join([_flat(x), _flat(coils), _flat(W)])
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    vals = np.array(out.stdout.split(), np.float64).reshape(-1, 2)
    vals = vals[:, 0] + 1j * vals[:, 1]
    nV = ny * nc * g.ntx
    V = vals[:nV].reshape(ny, nc, g.ntx)
    xa = vals[nV:].reshape(1, ny, nx)
    V_ref = np.transpose(O.hybrid_forward(g, coils, x)[:, 0], (1, 0, 2))  # [n][z][y][t] -> [y][n][t]
    assert np.linalg.norm(V - V_ref) < 1e-6 * np.linalg.norm(V_ref)
    xa_ref = O.hybrid_adjoint(g, coils, np.transpose(W, (1, 0, 2))[:, None])
    assert np.linalg.norm(xa - xa_ref) < 1e-6 * np.linalg.norm(xa_ref)
