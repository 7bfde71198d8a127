// Grouped Hermitian rank-k update of chi0 on the CUDA cores (Eq. 17, the
// "multi-u" form of Eq. 15): for every frequency w_j,
//   chi_GG'(w_j) += sum_p w_p(w_j) n_p(G) conj(n_p(G')),
// with the pair densities of one k-block stored pair-major, N[p][G].
//
// Used for the FP64 mode (DFMA) and the FP32 mode (FFMA).  Only tiles of the
// lower triangle are computed; the upper triangle is filled from it.  In the
// FP32 mode each thread folds its FP32 partial sums every 256 pairs into an
// FP32 (hi, lo) pair with Knuth's two-sum, and the result is added to the FP64
// chi0 once per k-block, so the rounding error does not grow with the number
// of pairs.
#include "rpa_internal.h"

namespace rpa {

constexpr int HT = 64;   // tile edge (complex elements)
constexpr int HK = 16;   // pairs per shared-memory stage

__global__ void pair_weights_kernel(const double* __restrict__ d, const double* __restrict__ df,
                                    const double* __restrict__ omega, int nw, int64_t P, double pref,
                                    double* __restrict__ w64, float* __restrict__ w32) {
  const int64_t total = (int64_t)nw * P;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(id / P);
    const int64_t p = id % P;
    const double dd = d[p];
    const double om = omega[j];
    const double w = pref * df[p] * 2.0 * dd / (om * om + dd * dd);
    if (w64) w64[id] = w;
    if (w32) w32[id] = (float)w;
  }
}

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += err;
}

__device__ __forceinline__ void tile_of(int t, int& ti, int& tj) {
  int i = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (i * (i + 1) / 2 > t) --i;
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  ti = i;
  tj = t - i * (i + 1) / 2;
}

template <typename T>
__global__ void __launch_bounds__(256) herk_simt_kernel(const c2<T>* __restrict__ N, int64_t P, int NG,
                                                        const T* __restrict__ wgt, double2* __restrict__ chi) {
  __shared__ c2<T> As[HK][HT];
  __shared__ c2<T> Bs[HK][HT];
  const int w = blockIdx.y;
  int ti, tj;
  tile_of(blockIdx.x, ti, tj);
  const int r0 = ti * HT, c0 = tj * HT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const T* wv = wgt + (int64_t)w * P;
  c2<T> acc[4][4];
  float hi[4][4][2], lo[4][4][2];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      acc[r][c] = mk<T>(0, 0);
      hi[r][c][0] = hi[r][c][1] = lo[r][c][0] = lo[r][c][1] = 0.f;
    }
  int since_fold = 0;
  // the next stage's elements are fetched into registers while the current
  // stage is multiplied
  constexpr int LQ = (HK * HT) / 256;
  c2<T> pa[LQ], pb[LQ];
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < LQ; ++q) {
      const int e = threadIdx.x + 256 * q;
      const int kk = e / HT, cc = e % HT;
      const int64_t p = k0 + kk;
      c2<T> a = mk<T>(0, 0), b = mk<T>(0, 0);
      if (p < P) {
        const T wp = wv[p];
        if (r0 + cc < NG) {
          a = N[p * NG + r0 + cc];
          a.x *= wp;
          a.y *= wp;
        }
        if (c0 + cc < NG) b = N[p * NG + c0 + cc];
      }
      pa[q] = a;
      pb[q] = b;
    }
  };
  // (FP32 only: the FP64 form is bound by the FP64 pipe and keeps its
  // registers for two resident blocks)
  constexpr bool PREFETCH = sizeof(T) == 4;
  if (PREFETCH) fetch(0);
  for (int64_t k0 = 0; k0 < P; k0 += HK) {
    if (!PREFETCH) fetch(k0);
#pragma unroll
    for (int q = 0; q < LQ; ++q) {
      const int e = threadIdx.x + 256 * q;
      As[e / HT][e % HT] = pa[q];
      Bs[e / HT][e % HT] = pb[q];
    }
    __syncthreads();
    if (PREFETCH && k0 + HK < P) fetch(k0 + HK);
#pragma unroll
    for (int kk = 0; kk < HK; ++kk) {
      c2<T> av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) av[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) cmac_cj<T>(acc[r][c], av[r], bv[c]);
    }
    __syncthreads();
    if (sizeof(T) == 4) {
      if (++since_fold == 16) {
        since_fold = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            two_sum_acc(hi[r][c][0], lo[r][c][0], (float)acc[r][c].x);
            two_sum_acc(hi[r][c][1], lo[r][c][1], (float)acc[r][c].y);
            acc[r][c] = mk<T>(0, 0);
          }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int row = r0 + ty + 16 * r, col = c0 + tx + 16 * c;
      if (row < NG && col < NG && row >= col) {
        double re, im;
        if (sizeof(T) == 4) {
          re = (double)hi[r][c][0] + (double)lo[r][c][0] + (double)acc[r][c].x;
          im = (double)hi[r][c][1] + (double)lo[r][c][1] + (double)acc[r][c].y;
        } else {
          re = (double)acc[r][c].x;
          im = (double)acc[r][c].y;
        }
        double2* dst = chi + ((int64_t)w * NG + row) * NG + col;
        double2 v = *dst;
        v.x += re;
        v.y += im;
        *dst = v;
      }
    }
}

static inline int gridn(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b > 152 * 64 ? 152 * 64 : (b < 1 ? 1 : b));
}

cudaError_t launch_pair_weights(const double* d, const double* df, const double* omega, int nw, int64_t P,
                                double pref, double* w64, float* w32, cudaStream_t s) {
  if ((int64_t)nw * P == 0) return cudaSuccess;
  pair_weights_kernel<<<gridn((int64_t)nw * P), 256, 0, s>>>(d, df, omega, nw, P, pref, w64, w32);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_herk_simt_w(const c2<T>* N, int64_t P, int NG, const T* wgt, int nw, double2* chi,
                               cudaStream_t s) {
  if (P == 0 || NG == 0 || nw == 0) return cudaSuccess;
  const int nt = (NG + HT - 1) / HT;
  dim3 grid(nt * (nt + 1) / 2, nw);
  herk_simt_kernel<T><<<grid, 256, 0, s>>>(N, P, NG, wgt, chi);
  return cudaGetLastError();
}

template cudaError_t launch_herk_simt_w<float>(const float2*, int64_t, int, const float*, int, double2*, cudaStream_t);
template cudaError_t launch_herk_simt_w<double>(const double2*, int64_t, int, const double*, int, double2*,
                                                cudaStream_t);

__global__ void hermitian_fill_kernel(double2* __restrict__ chi, int nw, int NG) {
  const int64_t total = (int64_t)nw * NG * NG;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(id % NG);
    const int64_t r = id / NG;
    const int i = (int)(r % NG);
    const int64_t w = r / NG;
    if (i < j) {
      const double2 v = chi[(w * NG + j) * NG + i];
      chi[id] = make_double2(v.x, -v.y);
    } else if (i == j) {
      chi[id].y = 0.0;
    }
  }
}

cudaError_t launch_hermitian_fill(double2* chi, int nw, int NG, cudaStream_t s) {
  const int64_t total = (int64_t)nw * NG * NG;
  if (total == 0) return cudaSuccess;
  hermitian_fill_kernel<<<gridn(total), 256, 0, s>>>(chi, nw, NG);
  return cudaGetLastError();
}

}  // namespace rpa
