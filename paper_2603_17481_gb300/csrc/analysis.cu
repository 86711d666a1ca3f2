// analysis.cu -- the carrier-phase kinetic-energy spectrum of Sec. 3.4 (the swarm's E(k)).
//
// The carrier phase is the liquid, chi = 1 where phi >= 1/2. The fluctuation u' = chi (u - <u>_liquid)
// is transformed per component with a cuFFT real-to-complex 3D transform (the library's FFT; the
// surrounding kernels are ours), and |u_hat|^2 / 2 with u_hat = FFT / N is summed into shells of
// |k| (k_a = 2 pi m_a / n_a, shell width 2 pi / max(n_a), shell floor(|k| / width + 1/2), with
// |k| / width = |(m_a max(n) / n_a)| exact on half-integer ties); the half spectrum counts twice except
// on the planes m_x = 0 and m_x = n_x / 2.
#include <cufft.h>

#include "launch.h"

namespace lbm {

namespace {

constexpr int kSpecThreads = 256;
constexpr int kSpecBlocks = 608;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums of chi u and chi over the box: per block, then one warp in a fixed order.
__global__ void __launch_bounds__(kSpecThreads)
k_liquid_mean_partial(const KParams P, const int32_t *__restrict__ phi, const float *__restrict__ u,
                      double *__restrict__ partials) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, c = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < P.N; n += stride) {
    if (phi_of(phi[n]) >= 0.5f) {
      s0 += u[n];
      s1 += u[P.N + n];
      s2 += u[2 * P.N + n];
      c += 1.0;
    }
  }
  __shared__ double sm[4][kSpecThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  s0 = warp_sum_d(s0); s1 = warp_sum_d(s1); s2 = warp_sum_d(s2); c = warp_sum_d(c);
  if (lane == 0) { sm[0][w] = s0; sm[1][w] = s1; sm[2][w] = s2; sm[3][w] = c; }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int k = 0; k < kSpecThreads / 32; k++) t += sm[threadIdx.x][k];
    partials[4 * blockIdx.x + threadIdx.x] = t;
  }
}

__global__ void k_liquid_mean_final(const double *__restrict__ partials, int n, double *__restrict__ mean) {
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = threadIdx.x; k < n; k += 32)
#pragma unroll
    for (int j = 0; j < 4; j++) a[j] += partials[4 * k + j];
#pragma unroll
  for (int j = 0; j < 4; j++) a[j] = warp_sum_d(a[j]);
  if (threadIdx.x == 0) {
    const double c = a[3] > 0.0 ? a[3] : 1.0;
    mean[0] = a[0] / c; mean[1] = a[1] / c; mean[2] = a[2] / c;
  }
}

// u'_a = chi (u_a - <u_a>), in FP32 for the transform.
__global__ void __launch_bounds__(kSpecThreads)
k_fluct(const KParams P, const int32_t *__restrict__ phi, const float *__restrict__ u, const double *__restrict__ mean,
        int a, float *__restrict__ out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const float m = (float)mean[a];
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < P.N; n += stride)
    out[n] = phi_of(phi[n]) >= 0.5f ? u[a * P.N + n] - m : 0.0f;
}

// Shell sums of the half spectrum (nx / 2 + 1 along x) of one component into this block's row of
// partials (nshells doubles per block, accumulated over the components).
__global__ void __launch_bounds__(kSpecThreads)
k_shells(const KParams P, const cufftComplex *__restrict__ uh, int nshells, double *__restrict__ partials) {
  extern __shared__ double hist[];
  for (int k = threadIdx.x; k < nshells; k += blockDim.x) hist[k] = 0.0;
  __syncthreads();
  const int nx = P.nx, ny = P.ny, nz = P.nz, hx = nx / 2 + 1;
  const double M = (double)max(nx, max(ny, nz));
  const double inv_n2 = 1.0 / ((double)P.N * (double)P.N);
  const long long total = (long long)hx * ny * nz;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += stride) {
    const int mx = (int)(e % hx), iy = (int)((e / hx) % ny), iz = (int)(e / ((long long)hx * ny));
    const int my = iy < (ny + 1) / 2 ? iy : iy - ny, mz = iz < (nz + 1) / 2 ? iz : iz - nz;
    const double kx = (double)mx * M / nx, ky = (double)my * M / ny, kz = (double)mz * M / nz;
    const int K = (int)floor(sqrt(kx * kx + ky * ky + kz * kz) + 0.5);  // ties round up
    if (K >= nshells) continue;
    const double w = (mx == 0 || (nx % 2 == 0 && mx == nx / 2)) ? 1.0 : 2.0;
    const cufftComplex v = uh[e];
    atomicAdd(&hist[K], 0.5 * w * ((double)v.x * v.x + (double)v.y * v.y) * inv_n2);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nshells; k += blockDim.x) partials[(long long)blockIdx.x * nshells + k] += hist[k];
}

__global__ void k_shells_final(const double *__restrict__ partials, int nblocks, int nshells, double *__restrict__ E) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nshells; k += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < nblocks; b++) t += partials[(long long)b * nshells + k];
    E[k] = t;
  }
}

}  // namespace

int spectrum_compute(const KParams &P, const int32_t *phi, const float *u, int nshells, double *E_dev,
                     cudaStream_t s) {
  if (nshells < 1 || nshells > kMaxSpectrumShells) return 1;
  const long long N = P.N;
  const long long nc = (long long)(P.nx / 2 + 1) * P.ny * P.nz;
  float *in = nullptr;
  cufftComplex *out = nullptr;
  double *part = nullptr, *mean = nullptr;
  cufftHandle plan = 0;
  bool have_plan = false;
  int rc = 0;
  cudaError_t e = cudaMalloc(&in, sizeof(float) * N);
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(cufftComplex) * nc);
  if (e == cudaSuccess) e = cudaMalloc(&part, sizeof(double) * ((size_t)kSpecBlocks * nshells + 4 * kSpecBlocks));
  if (e == cudaSuccess) e = cudaMalloc(&mean, sizeof(double) * 3);
  if (e == cudaSuccess) e = cudaMemsetAsync(part, 0, sizeof(double) * (size_t)kSpecBlocks * nshells, s);
  if (e != cudaSuccess) rc = 2;
  if (!rc) {
    const cufftResult r = P.nz > 1 ? cufftPlan3d(&plan, P.nz, P.ny, P.nx, CUFFT_R2C)
                                   : cufftPlan2d(&plan, P.ny, P.nx, CUFFT_R2C);
    if (r != CUFFT_SUCCESS) rc = 3;
    else have_plan = true;
  }
  if (!rc && cufftSetStream(plan, s) != CUFFT_SUCCESS) rc = 3;
  if (!rc) {
    double *mpart = part + (size_t)kSpecBlocks * nshells;
    k_liquid_mean_partial<<<kSpecBlocks, kSpecThreads, 0, s>>>(P, phi, u, mpart);
    k_liquid_mean_final<<<1, 32, 0, s>>>(mpart, kSpecBlocks, mean);
    for (int a = 0; a < (P.nz > 1 ? 3 : 2) && !rc; a++) {
      k_fluct<<<kSpecBlocks, kSpecThreads, 0, s>>>(P, phi, u, mean, a, in);
      if (cufftExecR2C(plan, in, out) != CUFFT_SUCCESS) rc = 3;
      else k_shells<<<kSpecBlocks, kSpecThreads, sizeof(double) * nshells, s>>>(P, out, nshells, part);
    }
    if (!rc) k_shells_final<<<(nshells + 255) / 256, 256, 0, s>>>(part, kSpecBlocks, nshells, E_dev);
    if (!rc && cudaGetLastError() != cudaSuccess) rc = 2;
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = 2;
  }
  if (have_plan) cufftDestroy(plan);
  cudaFree(in); cudaFree(out); cudaFree(part); cudaFree(mean);
  return rc;
}

}  // namespace lbm
