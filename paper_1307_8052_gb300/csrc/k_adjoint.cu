// Adjoint (reverse mode) of the chi0 / E_c path, for dE_c/dchi0 and the
// gradients with respect to the plane-wave coefficients C and projections P.
// Gradients follow the PyTorch complex convention g = 2 dE/d(conj z), so that
// dE = Re sum conj(g) dz.
//
//  * dE/dchi(q, w_j) = (w_q W_j / 2 pi) v^1/2 [1 - (1 - M_j)^-1] v^1/2
//    (derivative of Eqs. 1-2); (1 - M)^-1 = L^-H L^-1 from the FP64 Cholesky
//    factor by a blocked forward substitution and a Gram product.
//  * nbar_p = 2 sum_j w_p(w_j) Gamma_j n_p (adjoint of the rank-k update, Eq. 17).
//  * PAW (Eq. 6): gP_n += sum_m sum_G conj(nbar_nm) sum_j P_mj Q_ij, and
//    gP_m += sum_n sum_G nbar_nm conj(R_n(j,G)) with R_n(j,G) = sum_i conj(P_ni) Q_ij(G).
//  * Pair densities (Eq. 10): xbar(r) = (1/N_r) sum_G nbar(G) exp(+i (G+G0).r)
//    by the transposed pruned transforms, ubar_m += xbar u_n,
//    ubar_n += conj(xbar) u_m, and gC(Q) = sum_r exp(-i Q.r) ubar(r).
#include <algorithm>

#include "ff_math.cuh"
#include "rpa_internal.h"

namespace rpa {

static inline int gridx(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b > 152 * 64 ? 152 * 64 : (b < 1 ? 1 : b));
}

__host__ __device__ inline int pmod_a(int64_t a, int n) {
  int64_t r = a % n;
  return (int)(r < 0 ? r + n : r);
}

// ---------------------------------------------------------------- complex GEMM (FP64 or FP32)
// C[z] = beta C[z] + alpha opA(A[z]) B[z]; opA = 0: A is M x K (row-major, lda),
// opA = 1: A is stored K x M and used conjugate-transposed.
constexpr int ZT = 64, ZK = 16;

template <typename T>
__global__ void __launch_bounds__(256) zgemm_kernel(int M, int N, int K, c2<T> alpha, const c2<T>* __restrict__ A,
                                                    int64_t lda, int64_t sA, int opA, const c2<T>* __restrict__ B,
                                                    int64_t ldb, int64_t sB, c2<T> beta, c2<T>* __restrict__ C,
                                                    int64_t ldc, int64_t sC) {
  __shared__ c2<T> As[ZK][ZT];
  __shared__ c2<T> Bs[ZK][ZT];
  const int z = blockIdx.z;
  A += z * sA;
  B += z * sB;
  C += z * sC;
  const int m0 = blockIdx.y * ZT, n0 = blockIdx.x * ZT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  c2<T> acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = mk<T>(0, 0);
  for (int k0 = 0; k0 < K; k0 += ZK) {
#pragma unroll
    for (int q = 0; q < (ZK * ZT) / 256; ++q) {
      const int e = threadIdx.x + 256 * q;
      // A tile: element (row m0+r, k k0+kk)
      {
        const int r = e / ZK, kk = e % ZK;
        c2<T> v = mk<T>(0, 0);
        if (m0 + r < M && k0 + kk < K) {
          if (opA == 0) {
            v = A[(int64_t)(m0 + r) * lda + k0 + kk];
          } else {
            const c2<T> t = A[(int64_t)(k0 + kk) * lda + m0 + r];
            v = mk<T>(t.x, -t.y);
          }
        }
        As[kk][r] = v;
      }
      {
        const int kk = e / ZT, c = e % ZT;
        Bs[kk][c] = (k0 + kk < K && n0 + c < N) ? B[(int64_t)(k0 + kk) * ldb + n0 + c] : mk<T>(0, 0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < ZK; ++kk) {
      c2<T> a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) cmac<T>(acc[r][c], a[r], b[c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int m = m0 + ty + 16 * r, n = n0 + tx + 16 * c;
      if (m < M && n < N) {
        c2<T>* p = C + (int64_t)m * ldc + n;
        const c2<T> old = (beta.x == 0 && beta.y == 0) ? mk<T>(0, 0) : *p;
        const c2<T> a = acc[r][c];
        c2<T> v;
        v.x = beta.x * old.x - beta.y * old.y + alpha.x * a.x - alpha.y * a.y;
        v.y = beta.x * old.y + beta.y * old.x + alpha.x * a.y + alpha.y * a.x;
        *p = v;
      }
    }
}

template <typename T>
static cudaError_t launch_gemm_t(int M, int N, int K, c2<T> alpha, const c2<T>* A, int64_t lda, int64_t sA, int opA,
                                 const c2<T>* B, int64_t ldb, int64_t sB, c2<T> beta, c2<T>* C, int64_t ldc, int64_t sC,
                                 int batch, cudaStream_t s) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  dim3 grid((N + ZT - 1) / ZT, (M + ZT - 1) / ZT, batch);
  zgemm_kernel<T><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, opA, B, ldb, sB, beta, C, ldc, sC);
  return cudaGetLastError();
}

cudaError_t launch_zgemm(int M, int N, int K, double2 alpha, const double2* A, int64_t lda, int64_t sA, int opA,
                         const double2* B, int64_t ldb, int64_t sB, double2 beta, double2* C, int64_t ldc,
                         int64_t sC, int batch, cudaStream_t s) {
  return launch_gemm_t<double>(M, N, K, alpha, A, lda, sA, opA, B, ldb, sB, beta, C, ldc, sC, batch, s);
}

// W = Y^H Y for lower-triangular Y (Y = L^-1): W[i][j] = sum_{k >= max(i,j)}
// conj(Y[k][i]) Y[k][j].  Only lower-triangle 64 x 64 tiles of W are formed
// (W is Hermitian), each summing k from its first row (Y[k][i] = 0 for k < i).
__device__ __forceinline__ void lower_tile(int t, int& ti, int& tj) {
  int i = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (i * (i + 1) / 2 > t) --i;
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  ti = i;
  tj = t - i * (i + 1) / 2;
}

template <typename T>
__global__ void __launch_bounds__(256) yhy_lower_kernel(const c2<T>* __restrict__ Y, int n, c2<T>* __restrict__ W) {
  __shared__ c2<T> As[ZK][ZT];
  __shared__ c2<T> Bs[ZK][ZT];
  const int z = blockIdx.y;
  const c2<T>* Yz = Y + (int64_t)z * n * n;
  c2<T>* Wz = W + (int64_t)z * n * n;
  int ti, tj;
  lower_tile(blockIdx.x, ti, tj);
  const int m0 = ti * ZT, n0 = tj * ZT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  c2<T> acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = mk<T>(0, 0);
  for (int k0 = m0; k0 < n; k0 += ZK) {
#pragma unroll
    for (int q = 0; q < (ZK * ZT) / 256; ++q) {
      const int e = threadIdx.x + 256 * q;
      const int kk = e / ZT, c = e % ZT;
      const bool kin = k0 + kk < n;
      const c2<T> a = (kin && m0 + c < n) ? Yz[(int64_t)(k0 + kk) * n + m0 + c] : mk<T>(0, 0);
      As[kk][c] = mk<T>(a.x, -a.y);
      Bs[kk][c] = (kin && n0 + c < n) ? Yz[(int64_t)(k0 + kk) * n + n0 + c] : mk<T>(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < ZK; ++kk) {
      c2<T> a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) cmac<T>(acc[r][c], a[r], b[c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = m0 + ty + 16 * r, j = n0 + tx + 16 * c;
      if (i < n && j <= i) Wz[(int64_t)i * n + j] = acc[r][c];
    }
}

// ---------------------------------------------------------------- (1 - M)^-1 from the Cholesky factor
constexpr int FB = 32;

template <typename T>
__global__ void set_identity_kernel(c2<T>* __restrict__ Y, int n, int nw) {
  const int64_t total = (int64_t)nw * n * n;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total; id += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(id % n);
    const int i = (int)((id / n) % n);
    Y[id] = mk<T>(i == j ? 1 : 0, 0);
  }
}

// Y[i0 .. i0+b) <- L_ii^-1 Y[i0 .. i0+b), one column of Y per thread.
template <typename T>
__global__ void __launch_bounds__(256) fwd_sub_diag_kernel(const c2<T>* __restrict__ L, c2<T>* __restrict__ Y,
                                                           int n, int i0, int b) {
  __shared__ c2<T> Ld[FB][FB + 1];
  const int w = blockIdx.y;
  const c2<T>* Lw = L + (int64_t)w * n * n;
  c2<T>* Yw = Y + (int64_t)w * n * n;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int r = e / b, l = e % b;
    Ld[r][l] = (l <= r) ? Lw[(int64_t)(i0 + r) * n + i0 + l] : mk<T>(0, 0);
  }
  __syncthreads();
  // columns beyond the block are zero in these rows (Y is lower triangular)
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= i0 + b) return;
  c2<T> y[FB];
#pragma unroll
  for (int r = 0; r < FB; ++r) y[r] = (r < b) ? Yw[(int64_t)(i0 + r) * n + c] : mk<T>(0, 0);
#pragma unroll
  for (int r = 0; r < FB; ++r) {
    if (r < b) {
      c2<T> s = y[r];
#pragma unroll
      for (int l = 0; l < FB; ++l) {
        if (l < r) {
          const c2<T> a = Ld[r][l], x = y[l];
          s.x -= a.x * x.x - a.y * x.y;
          s.y -= a.x * x.y + a.y * x.x;
        }
      }
      const T d = (T)1 / Ld[r][r].x;
      y[r] = mk<T>(s.x * d, s.y * d);
    }
  }
#pragma unroll
  for (int r = 0; r < FB; ++r)
    if (r < b) Yw[(int64_t)(i0 + r) * n + c] = y[r];
}

// Gamma = c_w v^1/2 (I - W) v^1/2 (W = (1-M)^-1), stored as FP64 and optionally FP32.
__global__ void gamma_kernel(const double2* __restrict__ Wm, const double* __restrict__ v, const double* __restrict__ cw,
                             int n, int nw, double2* __restrict__ G64, float2* __restrict__ G32) {
  const int64_t total = (int64_t)nw * n * n;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total; id += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(id % n);
    const int64_t r = id / n;
    const int i = (int)(r % n);
    const int w = (int)(r / n);
    const double s = cw[w] * sqrt(v[i]) * sqrt(v[j]);
    const double2 x = Wm[id];
    // Hermitian part of (I - W); W is Hermitian up to rounding
    const double2 xt = Wm[((int64_t)w * n + j) * n + i];
    double re = -(0.5 * (x.x + xt.x)), im = -(0.5 * (x.y - xt.y));
    if (i == j) {
      re += 1.0;
      im = 0.0;
    }
    const double2 g = make_double2(s * re, s * im);
    if (G64) G64[id] = g;
    if (G32) G32[id] = make_float2((float)g.x, (float)g.y);
  }
}

// ---------------------------------------------------------------- float-float products of Gamma
// The two O(n^3) products of (1 - M)^-1 = L^-H L^-1 in float-float: inputs and
// outputs FP64, each FP64 element split into hi + lo FP32 on load, every
// complex multiply-add an exact FMA two-product with two-sum accumulation
// (about 44 significant bits; the FP32 pipe instead of the FP64 one).
// GRAM = false: C[z] = beta C[z] + alpha A[z] B[z] (A M x K, B K x N, row-major);
// with tri, B is lower triangular (B[k][j] = 0 for k < j), so a column tile
// starting at n0 sums k from n0.
// GRAM = true:  W[z] = Y^H Y on lower-triangle tiles, k from the tile's first
// row (Y lower triangular).
// A BM x (4096 / BM) tile per block of 256 threads, 4 x 4 outputs a thread;
// the FP64 elements of the next K slice are fetched into registers while the
// current slice (split into hi + lo in shared memory) is multiplied.
__device__ __forceinline__ void ffc_mac(float4& acc, float4 a, float4 b) {
  // re += a.re b.re - a.im b.im, im += a.re b.im + a.im b.re
  ff_mac(acc.x, acc.y, a.x, a.y, b.x, b.y);
  ff_mac(acc.x, acc.y, -a.z, -a.w, b.z, b.w);
  ff_mac(acc.z, acc.w, a.x, a.y, b.z, b.w);
  ff_mac(acc.z, acc.w, a.z, a.w, b.x, b.y);
}

template <bool GRAM, int BMt>
__global__ void __launch_bounds__(256) gemm_ff_kernel(int M, int N, int K, double2 alpha, const double2* __restrict__ A,
                                                      int64_t lda, int64_t sA, const double2* __restrict__ B,
                                                      int64_t ldb, int64_t sB, double2 beta, double2* __restrict__ C,
                                                      int64_t ldc, int64_t sC, int tri) {
  constexpr int BNt = 4096 / BMt;
  constexpr int TX = BNt / 4, TY = BMt / 4;  // thread grid TY x TX
  constexpr int LA = ZK * BMt / 256, LB = ZK * BNt / 256;
  static_assert(!GRAM || BMt == 64, "Gram tiles are square");
  __shared__ float4 As[ZK][BMt + 1];
  __shared__ float4 Bs[ZK][BNt];
  const int z = GRAM ? blockIdx.y : blockIdx.z;
  A += z * sA;
  B += z * sB;
  C += z * sC;
  int m0, n0, kbeg;
  if constexpr (GRAM) {
    int ti, tj;
    lower_tile(blockIdx.x, ti, tj);
    m0 = ti * BMt;
    n0 = tj * BNt;
    kbeg = m0;  // Y[k][i] = 0 for k < i
  } else {
    m0 = blockIdx.y * BMt;
    n0 = blockIdx.x * BNt;
    kbeg = tri ? n0 : 0;
  }
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  double2 pa[LA], pb[LB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = threadIdx.x + 256 * q;
      double2 a = make_double2(0.0, 0.0);
      if constexpr (GRAM) {
        // A = Y^H: element (i = m0 + c, k) = conj(Y[k][i]), threads along i
        const int kk = e / BMt, c = e % BMt;
        if (k0 + kk < K && m0 + c < M) {
          a = A[(int64_t)(k0 + kk) * lda + m0 + c];
          a.y = -a.y;
        }
      } else {
        // threads along k (rows of A are contiguous in k)
        const int r = e / ZK, kk = e % ZK;
        if (k0 + kk < K && m0 + r < M) a = A[(int64_t)(m0 + r) * lda + k0 + kk];
      }
      pa[q] = a;
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = threadIdx.x + 256 * q;
      const int kk = e / BNt, c = e % BNt;
      pb[q] = (k0 + kk < K && n0 + c < N) ? B[(int64_t)(k0 + kk) * ldb + n0 + c] : make_double2(0.0, 0.0);
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = threadIdx.x + 256 * q;
      if constexpr (GRAM)
        As[e / BMt][e % BMt] = ff_split(pa[q]);
      else
        As[e % ZK][e / ZK] = ff_split(pa[q]);
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = threadIdx.x + 256 * q;
      Bs[e / BNt][e % BNt] = ff_split(pb[q]);
    }
  };
  float4 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (kbeg < K) fetch(kbeg);
  for (int k0 = kbeg; k0 < K; k0 += ZK) {
    stash();
    __syncthreads();
    if (k0 + ZK < K) fetch(k0 + ZK);
#pragma unroll 4
    for (int kk = 0; kk < ZK; ++kk) {
      float4 a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + TY * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + TX * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) ffc_mac(acc[r][c], a[r], b[c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int m = m0 + ty + TY * r, n = n0 + tx + TX * c;
      if (m >= M || n >= N || (GRAM && n > m)) continue;
      double2* p = C + (int64_t)m * ldc + n;
      const double2 a = ff_to_double(acc[r][c]);
      const double2 old = (beta.x == 0.0 && beta.y == 0.0) ? make_double2(0.0, 0.0) : *p;
      double2 v;
      v.x = beta.x * old.x - beta.y * old.y + alpha.x * a.x - alpha.y * a.y;
      v.y = beta.x * old.y + beta.y * old.x + alpha.x * a.y + alpha.y * a.x;
      *p = v;
    }
}

// Gamma as run_gamma with its two products in float-float.
cudaError_t run_gamma_ff(const double2* L, const double* v, const double* cw, int nw, int n, double2* Y, double2* Wm,
                         double2* G64, float2* G32, cudaStream_t s, int64_t* launches) {
  cudaError_t e;
  int64_t nl = 0;
  set_identity_kernel<double><<<gridx((int64_t)nw * n * n), 256, 0, s>>>(Y, n, nw);
  ++nl;
  // right-looking: solve a panel of FB rows, then take its contribution out
  // of every row below it at once (a wide product with K = FB)
  for (int i0 = 0; i0 < n; i0 += FB) {
    const int b = (n - i0) < FB ? (n - i0) : FB;
    fwd_sub_diag_kernel<double><<<dim3((i0 + b + 63) / 64, nw), 64, 0, s>>>(L, Y, n, i0, b);
    ++nl;
    const int r0 = i0 + b;
    if (r0 < n) {
      // Y[r0:n, 0:r0] -= L[r0:n, i0:r0] Y[i0:r0, 0:r0]
      dim3 grid((r0 + 63) / 64, (n - r0 + 63) / 64, nw);
      gemm_ff_kernel<false, 64><<<grid, 256, 0, s>>>(n - r0, r0, b, make_double2(-1.0, 0.0),
                                                     L + (int64_t)r0 * n + i0, n, (int64_t)n * n, Y + (int64_t)i0 * n,
                                                     n, (int64_t)n * n, make_double2(1.0, 0.0), Y + (int64_t)r0 * n, n,
                                                     (int64_t)n * n, 0);
      ++nl;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const int nt = (n + 63) / 64;
  gemm_ff_kernel<true, 64><<<dim3(nt * (nt + 1) / 2, nw), 256, 0, s>>>(n, n, n, make_double2(1.0, 0.0), Y, n,
                                                                        (int64_t)n * n, Y, n, (int64_t)n * n,
                                                                        make_double2(0.0, 0.0), Wm, n, (int64_t)n * n,
                                                                        0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_hermitian_fill(Wm, nw, n, s)) != cudaSuccess) return e;
  gamma_kernel<<<gridx((int64_t)nw * n * n), 256, 0, s>>>(Wm, v, cw, n, nw, G64, G32);
  nl += 4;
  if (launches) *launches += nl;
  return cudaGetLastError();
}

// Mixed modes: L (FP64 lower factor) -> FP32 with a zero upper triangle.
__global__ void lower_to32_kernel(const double2* __restrict__ L, int n, int nw, float2* __restrict__ L32) {
  const int64_t total = (int64_t)nw * n * n;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total; id += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(id % n);
    const int i = (int)((id / n) % n);
    const double2 v = L[id];
    L32[id] = j <= i ? make_float2((float)v.x, (float)v.y) : make_float2(0.f, 0.f);
  }
}

// M = v^1/2 chi v^1/2 in FP32 as a full Hermitian matrix from the lower triangle of chi.
__global__ void m_from_chi_kernel(const double2* __restrict__ chi, const double* __restrict__ v, int n, int nw,
                                  float2* __restrict__ M) {
  const int64_t total = (int64_t)nw * n * n;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total; id += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(id % n);
    const int64_t r = id / n;
    const int i = (int)(r % n);
    const int w = (int)(r / n);
    const double sc = sqrt(v[i]) * sqrt(v[j]);
    double2 x;
    if (j <= i) {
      x = chi[id];
    } else {
      const double2 t = chi[((int64_t)w * n + j) * n + i];
      x = make_double2(t.x, -t.y);
    }
    M[id] = make_float2((float)(sc * x.x), (float)(sc * x.y));
  }
}

// W[i][j] = conj(W[j][i]) for j > i (FP32)
__global__ void hermitian_fill32_kernel(float2* __restrict__ W, int n, int nw) {
  const int64_t total = (int64_t)nw * n * n;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total; id += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(id % n);
    const int64_t r = id / n;
    const int i = (int)(r % n);
    const int w = (int)(r / n);
    if (j > i) {
      const float2 t = W[((int64_t)w * n + j) * n + i];
      W[id] = make_float2(t.x, -t.y);
    }
  }
}

// Gamma = c_w v^1/2 [I - (1 - M)^-1] v^1/2 = -c_w v^1/2 M (1 - M)^-1 v^1/2: from
// X = M W (W = (1 - M)^-1; X Hermitian in exact arithmetic), without the
// cancellation of I - W when M is small (high frequencies).
__global__ void gamma_mx_kernel(const float2* __restrict__ X, const double* __restrict__ v,
                                const double* __restrict__ cw, int n, int nw, double2* __restrict__ G64,
                                float2* __restrict__ G32) {
  const int64_t total = (int64_t)nw * n * n;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total; id += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(id % n);
    const int64_t r = id / n;
    const int i = (int)(r % n);
    const int w = (int)(r / n);
    const double s = -cw[w] * sqrt(v[i]) * sqrt(v[j]);
    const float2 x = X[id];
    const float2 xt = X[((int64_t)w * n + j) * n + i];
    double re = 0.5 * ((double)x.x + (double)xt.x), im = 0.5 * ((double)x.y - (double)xt.y);
    if (i == j) im = 0.0;
    const double2 g = make_double2(s * re, s * im);
    if (G64) G64[id] = g;
    if (G32) G32[id] = make_float2((float)g.x, (float)g.y);
  }
}

// The mixed-mode Gamma on the FP32 pipe: Y = L^-1 by the same blocked forward
// substitution, W = Y^H Y, X = M W, Gamma from X.  (1 - M) >= 1 (chi0 <= 0), so
// L has a unit-bounded inverse and FP32 keeps about 1e-6 relative accuracy.
// Scratch: Yb and Wb of nw n^2 complex FP64 each, used as two FP32 matrices
// apiece; G32 holds the FP32 factor until Gamma overwrites it.
cudaError_t run_gamma_mixed(const double2* L, const double2* chi, const double* v, const double* cw, int nw, int n,
                            double2* Yb, double2* Wb, double2* G64, float2* G32, cudaStream_t s, int64_t* launches) {
  cudaError_t e;
  int64_t nl = 0;
  const int64_t mat = (int64_t)nw * n * n;
  float2* Y = (float2*)Yb;
  float2* Mm = Y + mat;
  float2* W = (float2*)Wb;
  float2* X = W + mat;
  float2* L32 = G32;
  lower_to32_kernel<<<gridx(mat), 256, 0, s>>>(L, n, nw, L32);
  m_from_chi_kernel<<<gridx(mat), 256, 0, s>>>(chi, v, n, nw, Mm);
  set_identity_kernel<float><<<gridx(mat), 256, 0, s>>>(Y, n, nw);
  nl += 3;
  for (int i0 = 0; i0 < n; i0 += FB) {
    const int b = (n - i0) < FB ? (n - i0) : FB;
    if (i0 > 0) {
      if ((e = launch_gemm_t<float>(b, i0, i0, make_float2(-1.f, 0.f), L32 + (int64_t)i0 * n, n, (int64_t)n * n, 0,
                                    Y, n, (int64_t)n * n, make_float2(1.f, 0.f), Y + (int64_t)i0 * n, n,
                                    (int64_t)n * n, nw, s)) != cudaSuccess)
        return e;
      ++nl;
    }
    fwd_sub_diag_kernel<float><<<dim3((i0 + b + 63) / 64, nw), 64, 0, s>>>(L32, Y, n, i0, b);
    ++nl;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const int nt = (n + ZT - 1) / ZT;
  yhy_lower_kernel<float><<<dim3(nt * (nt + 1) / 2, nw), 256, 0, s>>>(Y, n, W);
  hermitian_fill32_kernel<<<gridx(mat), 256, 0, s>>>(W, n, nw);
  nl += 2;
  if ((e = launch_gemm_t<float>(n, n, n, make_float2(1.f, 0.f), Mm, n, (int64_t)n * n, 0, W, n, (int64_t)n * n,
                                make_float2(0.f, 0.f), X, n, (int64_t)n * n, nw, s)) != cudaSuccess)
    return e;
  gamma_mx_kernel<<<gridx(mat), 256, 0, s>>>(X, v, cw, n, nw, G64, G32);
  nl += 2;
  if (launches) *launches += nl;
  return cudaGetLastError();
}

cudaError_t run_gamma(const double2* L, const double* v, const double* cw, int nw, int n, double2* Y, double2* Wm,
                      double2* G64, float2* G32, cudaStream_t s, int64_t* launches) {
  cudaError_t e;
  int64_t nl = 0;
  set_identity_kernel<double><<<gridx((int64_t)nw * n * n), 256, 0, s>>>(Y, n, nw);
  ++nl;
  for (int i0 = 0; i0 < n; i0 += FB) {
    const int b = (n - i0) < FB ? (n - i0) : FB;
    if (i0 > 0) {
      // Y[i0:i0+b, 0:i0] -= L[i0:i0+b, 0:i0] Y[0:i0, 0:i0] (Y[0:i0, i0:] is zero)
      if ((e = launch_zgemm(b, i0, i0, make_double2(-1.0, 0.0), L + (int64_t)i0 * n, n, (int64_t)n * n, 0, Y, n,
                            (int64_t)n * n, make_double2(1.0, 0.0), Y + (int64_t)i0 * n, n, (int64_t)n * n, nw, s)) !=
          cudaSuccess)
        return e;
      ++nl;
    }
    fwd_sub_diag_kernel<double><<<dim3((i0 + b + 63) / 64, nw), 64, 0, s>>>(L, Y, n, i0, b);
    ++nl;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // W = Y^H Y = L^-H L^-1 = (1 - M)^-1: lower tiles, then the upper triangle by symmetry
  {
    const int nt = (n + ZT - 1) / ZT;
    yhy_lower_kernel<double><<<dim3(nt * (nt + 1) / 2, nw), 256, 0, s>>>(Y, n, Wm);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_hermitian_fill(Wm, nw, n, s)) != cudaSuccess) return e;
    nl += 2;
  }
  gamma_kernel<<<gridx((int64_t)nw * n * n), 256, 0, s>>>(Wm, v, cw, n, nw, G64, G32);
  nl += 2;
  if (launches) *launches += nl;
  return cudaGetLastError();
}

// ---------------------------------------------------------------- nbar = 2 sum_w w_p(w) Gamma_w n_p
// Nbar[p][G] = 2 sum_w wgt[w][p] sum_G' Gamma_w[G][G'] N[p][G'] = 2 sum_(w,G') A[p][(w,G')] conj(Gamma_w[G'][G]).
template <typename T>
__global__ void __launch_bounds__(256) nbar_kernel(const c2<T>* __restrict__ N, int64_t P, int NG,
                                                   const T* __restrict__ wgt, const c2<T>* __restrict__ Gam, int nw,
                                                   c2<T>* __restrict__ Nbar) {
  __shared__ c2<T> As[ZK][ZT];
  __shared__ c2<T> Bs[ZK][ZT];
  const int64_t p0 = (int64_t)blockIdx.y * ZT;
  const int g0 = blockIdx.x * ZT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  c2<T> acc[4][4];
  double hi[4][4][2];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      acc[r][c] = mk<T>(0, 0);
      hi[r][c][0] = hi[r][c][1] = 0.0;
    }
  for (int w = 0; w < nw; ++w) {
    const c2<T>* Gw = Gam + (int64_t)w * NG * NG;
    const T* ww = wgt + (int64_t)w * P;
    for (int k0 = 0; k0 < NG; k0 += ZK) {
#pragma unroll
      for (int q = 0; q < (ZK * ZT) / 256; ++q) {
        const int e = threadIdx.x + 256 * q;
        {
          const int r = e / ZK, kk = e % ZK;
          const int64_t p = p0 + r;
          c2<T> a = mk<T>(0, 0);
          if (p < P && k0 + kk < NG) {
            a = N[p * NG + k0 + kk];
            const T s = ww[p];
            a.x *= s;
            a.y *= s;
          }
          As[kk][r] = a;
        }
        {
          const int kk = e / ZT, c = e % ZT;
          c2<T> b = mk<T>(0, 0);
          if (k0 + kk < NG && g0 + c < NG) {
            b = Gw[(int64_t)(k0 + kk) * NG + g0 + c];
            b.y = -b.y;
          }
          Bs[kk][c] = b;
        }
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < ZK; ++kk) {
        c2<T> a[4], b[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
        for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) cmac<T>(acc[r][c], a[r], b[c]);
      }
      __syncthreads();
    }
    // fold each frequency's partial into FP64 so FP32 rounding does not grow with nw
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        hi[r][c][0] += (double)acc[r][c].x;
        hi[r][c][1] += (double)acc[r][c].y;
        acc[r][c] = mk<T>(0, 0);
      }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t p = p0 + ty + 16 * r;
      const int g = g0 + tx + 16 * c;
      if (p < P && g < NG) Nbar[p * NG + g] = mk<T>((T)(2.0 * hi[r][c][0]), (T)(2.0 * hi[r][c][1]));
    }
}

template <typename T>
cudaError_t launch_nbar(const c2<T>* N, int64_t P, int NG, const T* wgt, const c2<T>* Gam, int nw, c2<T>* Nbar,
                        cudaStream_t s) {
  if (P == 0) return cudaSuccess;
  dim3 grid((NG + ZT - 1) / ZT, (unsigned)((P + ZT - 1) / ZT));
  nbar_kernel<T><<<grid, 256, 0, s>>>(N, P, NG, wgt, Gam, nw, Nbar);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- PAW adjoint
// Y[aL][kp][G] = sum_b conj(Nbar[(aL, b)][G]) Pm[b][kp]
template <typename T>
__global__ void paw_adj_y_kernel(const c2<T>* __restrict__ Nbar, int nL, int nR, int NG, const c2<T>* __restrict__ Pm,
                                 int KP, c2<T>* __restrict__ Y) {
  const int64_t total = (int64_t)nL * KP * NG;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total; id += (int64_t)gridDim.x * blockDim.x) {
    const int ig = (int)(id % NG);
    const int64_t r = id / NG;
    const int kp = (int)(r % KP);
    const int a = (int)(r / KP);
    c2<T> acc = mk<T>(0, 0);
    const c2<T>* nb = Nbar + (int64_t)a * nR * NG + ig;
    for (int b = 0; b < nR; ++b) cmac<T>(acc, mk<T>(nb[(int64_t)b * NG].x, -nb[(int64_t)b * NG].y), Pm[(int64_t)b * KP + kp]);
    Y[id] = acc;
  }
}

// gPk[Lidx[aL]][kp_i] += sum_j sum_G Q^a_ij(G) Y[aL][(a,j)][G]   (one block per (aL, kp_i))
template <typename T>
__global__ void __launch_bounds__(256) paw_adj_pk_kernel(const c2<T>* __restrict__ Y, int NG, int KP,
                                                         const double2* __restrict__ Q, const int* __restrict__ atom_of_kp,
                                                         const int* __restrict__ idx_in_atom,
                                                         const int* __restrict__ atom_off,
                                                         const int64_t* __restrict__ q_off,
                                                         const int* __restrict__ nproj, const int* __restrict__ Lidx,
                                                         double2* __restrict__ gP) {
  __shared__ double red[2][256];
  const int kpi = blockIdx.x % KP;
  const int aL = blockIdx.x / KP;
  const int atom = atom_of_kp[kpi];
  const int i = idx_in_atom[kpi];
  const int ni = nproj[atom];
  double sx = 0.0, sy = 0.0;
  for (int j = 0; j < ni; ++j) {
    const c2<T>* y = Y + ((int64_t)aL * KP + atom_off[atom] + j) * NG;
    const double2* qij = Q + q_off[atom] + ((int64_t)i * ni + j) * NG;
    for (int g = threadIdx.x; g < NG; g += blockDim.x) {
      const double2 q = qij[g];
      const c2<T> yy = y[g];
      sx += q.x * (double)yy.x - q.y * (double)yy.y;
      sy += q.x * (double)yy.y + q.y * (double)yy.x;
    }
  }
  red[0][threadIdx.x] = sx;
  red[1][threadIdx.x] = sy;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double2* dst = gP + (int64_t)Lidx[aL] * KP + kpi;
    dst->x += red[0][0];
    dst->y += red[1][0];
  }
}

// gPkp as a tiled product: for occupied band aL (grid z), part[aL][b][kp] =
// sum_G Nbar[(aL, b)][G] conj(R[aL][kp][G]) over 32 b x 64 kp tiles, products
// summed in T over G slices (32 in FP32, 16 in FP64) and the slices in FP64;
// paw_adj_pkp_reduce adds the bands in order to gP[Ridx[b]].
template <typename T>
__global__ void __launch_bounds__(256) paw_adj_pkp_tile_kernel(const c2<T>* __restrict__ Nbar,
                                                               const c2<T>* __restrict__ R, int nR, int NG, int KP,
                                                               double2* __restrict__ part) {
  constexpr int KT = sizeof(T) == 4 ? 32 : 16;
  __shared__ c2<T> As[KT][33];
  __shared__ c2<T> Bs[KT][65];
  const int aL = blockIdx.z;
  const int b0 = blockIdx.x * 32, k0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const c2<T>* nb = Nbar + ((int64_t)aL * nR) * NG;
  const c2<T>* rr = R + ((int64_t)aL * KP) * NG;
  double2 acc[2][4];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_double2(0.0, 0.0);
  for (int g0 = 0; g0 < NG; g0 += KT) {
#pragma unroll
    for (int q = 0; q < 32 * KT / 256; ++q) {
      const int e = threadIdx.x + 256 * q, bb = e / KT, kk = e % KT;
      As[kk][bb] = (b0 + bb < nR && g0 + kk < NG) ? nb[(int64_t)(b0 + bb) * NG + g0 + kk] : mk<T>(0, 0);
    }
#pragma unroll
    for (int q = 0; q < 64 * KT / 256; ++q) {
      const int e = threadIdx.x + 256 * q, cc = e / KT, kk = e % KT;
      Bs[kk][cc] = (k0 + cc < KP && g0 + kk < NG) ? rr[(int64_t)(k0 + cc) * NG + g0 + kk] : mk<T>(0, 0);
    }
    __syncthreads();
    c2<T> s[2][4];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) s[r][c] = mk<T>(0, 0);
#pragma unroll 8
    for (int kk = 0; kk < KT; ++kk) {
      c2<T> a[2], bv[4];
#pragma unroll
      for (int r = 0; r < 2; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) cmac_cj<T>(s[r][c], a[r], bv[c]);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        acc[r][c].x += (double)s[r][c].x;
        acc[r][c].y += (double)s[r][c].y;
      }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int b = b0 + ty + 16 * r, kp = k0 + tx + 16 * c;
      if (b < nR && kp < KP) part[((int64_t)aL * nR + b) * KP + kp] = acc[r][c];
    }
}

// gP[Ridx[b]][kp] += sum_aL part[aL][b][kp], bands in order
__global__ void paw_adj_pkp_reduce_kernel(const double2* __restrict__ part, int nL, int nR, int KP,
                                          const int* __restrict__ Ridx, double2* __restrict__ gP) {
  const int64_t total = (int64_t)nR * KP;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total; id += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(id / KP), kp = (int)(id % KP);
    double sx = 0.0, sy = 0.0;
    for (int aL = 0; aL < nL; ++aL) {
      const double2 v = part[(int64_t)aL * total + id];
      sx += v.x;
      sy += v.y;
    }
    double2* dst = gP + (int64_t)Ridx[b] * KP + kp;
    dst->x += sx;
    dst->y += sy;
  }
}

template <typename T>
cudaError_t launch_paw_adjoint(const c2<T>* Nbar, const c2<T>* R, const c2<T>* Pm, int nL, int nR, int NG, int KP,
                               const double2* Q, const int* atom_of_kp, const int* idx_in_atom, const int* atom_off,
                               const int64_t* q_off, const int* nproj, const int* Lidx, const int* Ridx, c2<T>* Ywork,
                               double2* part, double2* gPk, double2* gPkp, cudaStream_t s) {
  if ((int64_t)nL * nR * KP == 0) return cudaSuccess;
  paw_adj_y_kernel<T><<<gridx((int64_t)nL * KP * NG), 256, 0, s>>>(Nbar, nL, nR, NG, Pm, KP, Ywork);
  paw_adj_pk_kernel<T><<<nL * KP, 256, 0, s>>>(Ywork, NG, KP, Q, atom_of_kp, idx_in_atom, atom_off, q_off, nproj,
                                                Lidx, gPk);
  paw_adj_pkp_tile_kernel<T><<<dim3((nR + 31) / 32, (KP + 63) / 64, nL), 256, 0, s>>>(Nbar, R, nR, NG, KP, part);
  paw_adj_pkp_reduce_kernel<<<gridx((int64_t)nR * KP), 256, 0, s>>>(part, nL, nR, KP, Ridx, gPkp);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- pair-density adjoint
// Stage C^T: T2bar[pl][o1][o2][j3] = (1/N_r) sum_{G in column (o1,o2)} Nbar[p][G] exp(+2 pi i g3 j3 / N3).
// Column lists: col_start[n1*n2+1], col_g[k] = sphere index, col_g3[k] = g3 mod N3 of that point.
// Chunk pl -> pair p = p0 + (pl / mc) nR + pl % mc: mc consecutive unoccupied
// bands of np / mc consecutive occupied bands.  With tab the twiddles sit in
// shared memory as a table over (g3 mod N3, j3), so no term takes a modulus.
template <typename T>
__global__ void __launch_bounds__(256) adj_stageC_kernel(const c2<T>* __restrict__ Nbar, int NG, int64_t p0, int np,
                                                         int mc, int nR, int ncol, int N3,
                                                         const int* __restrict__ col_start,
                                                         const int* __restrict__ col_g, const int* __restrict__ col_g3,
                                                         double inv_nr, int tab, const c2<T>* __restrict__ twg,
                                                         c2<T>* __restrict__ T2) {
  extern __shared__ unsigned char smem_raw[];
  c2<T>* tw1 = reinterpret_cast<c2<T>*>(smem_raw);  // exp(2 pi i t / N3), t < N3
  c2<T>* tw = tab ? tw1 + N3 : tw1;                   // tab: [g3 mod N3][j3]
  for (int e = threadIdx.x; e < N3; e += blockDim.x) {
    if (twg) {
      tw1[e] = twg[e];  // the same values, formed once per block of pairs
    } else {
      double sn, cs;
      sincospi(2.0 * (double)e / (double)N3, &sn, &cs);
      tw1[e] = mk<T>((T)cs, (T)sn);
    }
  }
  __syncthreads();
  if (tab) {
    for (int e = threadIdx.x; e < N3 * N3; e += blockDim.x) tw[e] = tw1[((e / N3) * (e % N3)) % N3];
    __syncthreads();
  }
  const int64_t total = (int64_t)np * ncol * N3;
  const T scale = (T)inv_nr;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total; id += (int64_t)gridDim.x * blockDim.x) {
    const int j3 = (int)(id % N3);
    const int64_t r = id / N3;
    const int col = (int)(r % ncol);
    const int pl = (int)(r / ncol);
    const c2<T>* nb = Nbar + (p0 + (int64_t)(pl / mc) * nR + pl % mc) * NG;
    c2<T> acc = mk<T>(0, 0);
    const int kb = col_start[col], ke = col_start[col + 1];
    if (tab) {
      for (int k = kb; k < ke; ++k) cmac<T>(acc, nb[col_g[k]], tw[col_g3[k] * N3 + j3]);
    } else {
      for (int k = kb; k < ke; ++k) cmac<T>(acc, nb[col_g[k]], tw[(col_g3[k] * j3) % N3]);
    }
    acc.x *= scale;
    acc.y *= scale;
    T2[id] = acc;
  }
}

template <typename T>
cudaError_t launch_adj_stageC(const c2<T>* Nbar, int NG, int64_t p0, int np, int mc, int nR, int ncol, int N3,
                              const int* col_start, const int* col_g, const int* col_g3, double inv_nr,
                              const c2<T>* tw3, c2<T>* T2, cudaStream_t s) {
  const int64_t total = (int64_t)np * ncol * N3;
  if (total == 0) return cudaSuccess;
  if (mc < 1 || np % mc) return cudaErrorInvalidValue;
  const int tab = (int64_t)N3 * (N3 + 1) * sizeof(c2<T>) <= 48 * 1024 ? 1 : 0;
  const size_t smem = (tab ? (size_t)N3 * (N3 + 1) : (size_t)N3) * sizeof(c2<T>);
  // a grid of eight blocks per SM amortises the table over many outputs
  const int grid = std::min(gridx(total), 152 * 8);
  adj_stageC_kernel<T><<<grid, 256, smem, s>>>(Nbar, NG, p0, np, mc, nR, ncol, N3, col_start, col_g, col_g3, inv_nr,
                                               tab, tw3, T2);
  return cudaGetLastError();
}

// Stage A^T with the products: for the chunk's pairs (all with the same occupied
// band n), xbar[pl][j1][j23] = sum_o1 T1bar[pl][o1][j23] exp(+2 pi i g1 j1 / N1);
// ubar_m[j] += xbar u_n[j] (distinct m per pair: no race) and xbar is kept for
// the ubar_n reduction.  The twiddle table is tw[o1][j1] (FP64-accurate).
template <typename T>
__global__ void __launch_bounds__(256) adj_stageA_kernel(const c2<T>* __restrict__ T1, int np, int n1, int N1, int N23,
                                                         const c2<T>* __restrict__ tw, const c2<T>* __restrict__ Un,
                                                         const c2<T>* __restrict__ Ukp, const int* __restrict__ Ridx,
                                                         int nR, int64_t p0, c2<T>* __restrict__ Ubar_kp,
                                                         c2<T>* __restrict__ Xbar) {
  const int64_t Nr = (int64_t)N1 * N23;
  const int64_t total = (int64_t)np * N23;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total; id += (int64_t)gridDim.x * blockDim.x) {
    const int j23 = (int)(id % N23);
    const int pl = (int)(id / N23);
    const int m = Ridx[(p0 + pl) % nR];
    const c2<T>* src = T1 + (int64_t)pl * n1 * N23 + j23;
    for (int j1 = 0; j1 < N1; ++j1) {
      c2<T> x = mk<T>(0, 0);
      for (int o = 0; o < n1; ++o) cmac<T>(x, src[(int64_t)o * N23], tw[o * N1 + j1]);
      const int64_t jj = (int64_t)j1 * N23 + j23;
      Xbar[(int64_t)pl * Nr + jj] = x;
      c2<T>* ub = Ubar_kp + (int64_t)m * Nr + jj;
      c2<T> v = *ub;
      cmac<T>(v, x, Un[jj]);
      *ub = v;
    }
  }
}

template <typename T>
cudaError_t launch_adj_stageA(const c2<T>* T1, int np, int n1, int N1, int N23, const c2<T>* tw, const c2<T>* Un,
                              const c2<T>* Ukp, const int* Ridx, int nR, int64_t p0, c2<T>* Ubar_kp, c2<T>* Xbar,
                              cudaStream_t s) {
  const int64_t total = (int64_t)np * N23;
  if (total == 0) return cudaSuccess;
  adj_stageA_kernel<T><<<gridx(total), 256, 0, s>>>(T1, np, n1, N1, N23, tw, Un, Ukp, Ridx, nR, p0, Ubar_kp, Xbar);
  return cudaGetLastError();
}

// ubar_n[j] += sum_pl conj(xbar[pl][j]) u_m(pl)[j]   (thread per grid point)
template <typename T>
__global__ void adj_un_kernel(const c2<T>* __restrict__ Xbar, int np, int64_t Nr, const c2<T>* __restrict__ Ukp,
                              const int* __restrict__ Ridx, int nR, int64_t p0, c2<T>* __restrict__ Ubar_n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < Nr; j += (int64_t)gridDim.x * blockDim.x) {
    c2<T> acc = Ubar_n[j];
    for (int pl = 0; pl < np; ++pl) {
      const c2<T> x = Xbar[(int64_t)pl * Nr + j];
      const c2<T> u = Ukp[(int64_t)Ridx[(p0 + pl) % nR] * Nr + j];
      // conj(x) * u
      acc.x += x.x * u.x + x.y * u.y;
      acc.y += x.x * u.y - x.y * u.x;
    }
    Ubar_n[j] = acc;
  }
}

template <typename T>
cudaError_t launch_adj_un(const c2<T>* Xbar, int np, int64_t Nr, const c2<T>* Ukp, const int* Ridx, int nR, int64_t p0,
                          c2<T>* Ubar_n, cudaStream_t s) {
  if (Nr == 0 || np == 0) return cudaSuccess;
  adj_un_kernel<T><<<gridx(Nr), 256, 0, s>>>(Xbar, np, Nr, Ukp, Ridx, nR, p0, Ubar_n);
  return cudaGetLastError();
}

// Stage A^T fused with both products, x-bar never stored: a chunk holds the
// pairs (a0 + i, m0 + j), i < A occupied bands, j < mc unoccupied bands, as
// T1[i mc + j][o1][j23].  A block owns 32 columns j23 (one per lane) and a
// slice of the chunk's m; warp w owns the rows j1 = w, w + 4, ... .  Per pair
// and row: x_i = sum_o1 T1[o1] tw[o1][j1]; ubar_m[j] += sum_i x_i u_{a0+i}[j]
// (one read-modify-write per m and row for all A bands; distinct m per thread:
// no race); the u_n terms conj(x_i) u_m[j] are summed over the block's m in
// shared memory and written once per block as part[slice][i][j], which
// adj_part_reduce adds to ubar_n in slice order (deterministic).
constexpr int ADJA_WARPS = 4;

template <typename T, int NI, int A>
__global__ void __launch_bounds__(128) adj_stageA_fused_kernel(const c2<T>* __restrict__ T1, int mc, int n1, int N1,
                                                               int N23, const c2<T>* __restrict__ tw,
                                                               const c2<T>* __restrict__ Un0,
                                                               const c2<T>* __restrict__ Un1,
                                                               const c2<T>* __restrict__ Ukp,
                                                               const int* __restrict__ Ridx, int m0,
                                                               c2<T>* __restrict__ Ubar_kp, c2<T>* __restrict__ part) {
  extern __shared__ unsigned char smem_raw[];
  c2<T>* tws = reinterpret_cast<c2<T>*>(smem_raw);  // [N1][NI], o1 beyond n1 zero
  c2<T>* uns = tws + N1 * NI;                        // [A][N1][32] u_n of the block's columns
  c2<T>* accs = uns + A * N1 * 32;                   // [A][N1][32] u_n terms of the block's m
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j23 = blockIdx.x * 32 + lane;
  const int64_t Nr = (int64_t)N1 * N23;
  for (int e = threadIdx.x; e < N1 * NI; e += blockDim.x) {
    const int j1 = e / NI, o = e % NI;
    tws[e] = o < n1 ? tw[o * N1 + j1] : mk<T>(0, 0);
  }
  for (int e = threadIdx.x; e < A * N1 * 32; e += blockDim.x) {
    const int i = e / (N1 * 32), r = e % (N1 * 32), j1 = r >> 5, l = r & 31;
    const int jj = blockIdx.x * 32 + l;
    const c2<T>* un = i ? Un1 : Un0;
    uns[e] = jj < N23 ? un[(int64_t)j1 * N23 + jj] : mk<T>(0, 0);
    accs[e] = mk<T>(0, 0);
  }
  __syncthreads();
  const int per = (mc + gridDim.y - 1) / gridDim.y;
  const int jb = blockIdx.y * per, je = min(mc, jb + per);
  if (j23 < N23) {
    for (int j = jb; j < je; ++j) {
      const int m = Ridx[m0 + j];
      c2<T> t[A][NI];
#pragma unroll
      for (int i = 0; i < A; ++i) {
        const c2<T>* src = T1 + ((int64_t)(i * mc + j) * n1) * N23 + j23;
#pragma unroll
        for (int o = 0; o < NI; ++o) t[i][o] = o < n1 ? src[(int64_t)o * N23] : mk<T>(0, 0);
      }
      const c2<T>* um = Ukp + (int64_t)m * Nr + j23;
      c2<T>* ubm = Ubar_kp + (int64_t)m * Nr + j23;
#pragma unroll 2
      for (int j1 = warp; j1 < N1; j1 += ADJA_WARPS) {
        const int64_t off = (int64_t)j1 * N23;
        const c2<T> u = um[off];
        c2<T> v = ubm[off];
        const c2<T>* twj = tws + j1 * NI;
#pragma unroll
        for (int i = 0; i < A; ++i) {
          c2<T> x = mk<T>(0, 0);
#pragma unroll
          for (int o = 0; o < NI; ++o) cmac<T>(x, t[i][o], twj[o]);
          cmac<T>(v, x, uns[(i * N1 + j1) * 32 + lane]);
          c2<T>& acc = accs[(i * N1 + j1) * 32 + lane];  // row j1 belongs to this warp alone
          const c2<T> cu = cj_mul<T>(x, u);
          acc.x += cu.x;
          acc.y += cu.y;
        }
        ubm[off] = v;
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < A * N1 * 32; e += blockDim.x) {
    const int i = e / (N1 * 32), r = e % (N1 * 32), j1 = r >> 5, l = r & 31;
    const int jj = blockIdx.x * 32 + l;
    if (jj < N23) part[((int64_t)blockIdx.y * A + i) * Nr + (int64_t)j1 * N23 + jj] = accs[e];
  }
}

// ubar_n_i[j] += sum_s part[s][i][j], slices in order
template <typename T>
__global__ void adj_part_reduce_kernel(const c2<T>* __restrict__ part, int S, int A, int64_t Nr, c2<T>* __restrict__ Ub0,
                                       c2<T>* __restrict__ Ub1) {
  const int64_t total = (int64_t)A * Nr;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total; id += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(id / Nr);
    const int64_t j = id % Nr;
    c2<T>* ub = (i ? Ub1 : Ub0) + j;
    c2<T> acc = *ub;
    for (int sl = 0; sl < S; ++sl) {
      const c2<T> v = part[((int64_t)sl * A + i) * Nr + j];
      acc.x += v.x;
      acc.y += v.y;
    }
    *ub = acc;
  }
}

template <typename T>
size_t adj_stageA_fused_smem(int N1, int n1, int A) {
  const int ni = n1 <= 8 ? 8 : n1 <= 12 ? 12 : n1 <= 14 ? 14 : 16;
  return sizeof(c2<T>) * ((size_t)N1 * ni + 2 * (size_t)A * N1 * 32);
}

// Slices of the chunk's m per column tile: about four blocks per SM in all.
int adj_stageA_fused_slices(int mc, int N23) {
  const int gx = (N23 + 31) / 32;
  return std::max(1, std::min(mc, (4 * 152 + gx - 1) / gx));
}

template <typename T, int NI, int A>
static cudaError_t adj_fused_launch(const c2<T>* T1, int mc, int n1, int N1, int N23, const c2<T>* tw,
                                    const c2<T>* Un0, const c2<T>* Un1, const c2<T>* Ukp, const int* Ridx, int m0,
                                    c2<T>* Ubar_kp, c2<T>* part, int S, size_t smem, cudaStream_t s) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(adj_stageA_fused_kernel<T, NI, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  adj_stageA_fused_kernel<T, NI, A><<<dim3((N23 + 31) / 32, S), 32 * ADJA_WARPS, smem, s>>>(
      T1, mc, n1, N1, N23, tw, Un0, Un1, Ukp, Ridx, m0, Ubar_kp, part);
  return cudaGetLastError();
}

// A in {1, 2}, n1 <= 16, shared memory within 200 KB (adj_stageA_fused_smem);
// part holds S * A * N1 * N23 elements, S = adj_stageA_fused_slices(mc, N23).
template <typename T>
cudaError_t launch_adj_stageA_fused(const c2<T>* T1, int A, int mc, int n1, int N1, int N23, const c2<T>* tw,
                                    const c2<T>* Un0, const c2<T>* Un1, const c2<T>* Ukp, const int* Ridx, int m0,
                                    c2<T>* Ubar_kp, c2<T>* Ubar_n0, c2<T>* Ubar_n1, c2<T>* part, cudaStream_t s) {
  if (mc == 0 || N23 == 0 || N1 == 0) return cudaSuccess;
  const size_t smem = adj_stageA_fused_smem<T>(N1, n1, A);
  if ((A != 1 && A != 2) || n1 < 1 || n1 > 16 || smem > 200 * 1024) return cudaErrorInvalidValue;
  const int S = adj_stageA_fused_slices(mc, N23);
  cudaError_t e;
#define ADJA_CASE(NI_)                                                                                          \
  e = A == 2 ? adj_fused_launch<T, NI_, 2>(T1, mc, n1, N1, N23, tw, Un0, Un1, Ukp, Ridx, m0, Ubar_kp, part, S, smem, s) \
             : adj_fused_launch<T, NI_, 1>(T1, mc, n1, N1, N23, tw, Un0, Un0, Ukp, Ridx, m0, Ubar_kp, part, S, smem, s)
  if (n1 <= 8) ADJA_CASE(8);
  else if (n1 <= 12) ADJA_CASE(12);
  else if (n1 <= 14) ADJA_CASE(14);
  else ADJA_CASE(16);
#undef ADJA_CASE
  if (e != cudaSuccess) return e;
  const int64_t Nr = (int64_t)N1 * N23;
  adj_part_reduce_kernel<T><<<gridx(A * Nr), 256, 0, s>>>(part, S, A, Nr, Ubar_n0, A == 2 ? Ubar_n1 : Ubar_n0);
  return cudaGetLastError();
}

// Twiddles of the transposed transforms: tw[jc][o][jj] = exp(+2 pi i (lo + o)(16 jc + jj) / N)
// (layout of the stage-B kernel with input axis o and 16 outputs j per chunk), and
// the plain matrix tw[o][j] used by stage A^T.
template <typename T>
__global__ void twiddle_adj_kernel(c2<T>* __restrict__ tw, int N, int lo, int nin, int chunked) {
  const int nch = (N + 15) / 16;
  const int64_t total = chunked ? (int64_t)nch * nin * 16 : (int64_t)nin * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int o, j;
    if (chunked) {
      const int jc = (int)(e / ((int64_t)nin * 16));
      const int r = (int)(e % ((int64_t)nin * 16));
      o = r / 16;
      j = jc * 16 + r % 16;
    } else {
      o = (int)(e / N);
      j = (int)(e % N);
    }
    if (j < N) {
      const int t = pmod_a((int64_t)(lo + o) * j, N);
      double s, c;
      sincospi(2.0 * (double)t / (double)N, &s, &c);
      tw[e] = mk<T>((T)c, (T)s);
    } else {
      tw[e] = mk<T>(0, 0);
    }
  }
}

template <typename T>
cudaError_t launch_twiddle_adj(c2<T>* tw, int N, int lo, int nin, int chunked, cudaStream_t s) {
  const int64_t total = chunked ? (int64_t)((N + 15) / 16) * nin * 16 : (int64_t)nin * N;
  twiddle_adj_kernel<T><<<gridx(total), 256, 0, s>>>(tw, N, lo, nin, chunked);
  return cudaGetLastError();
}

// Gather a Miller box back onto the plane-wave list and accumulate in FP64:
// dC[b][q] += box[b][pos[q]].
template <typename T>
__global__ void gather_box_kernel(const c2<T>* __restrict__ box, int nb, int npw, const int* __restrict__ pos,
                                  int64_t boxsz, double2* __restrict__ dC) {
  const int64_t total = (int64_t)nb * npw;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total; id += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(id / npw), q = (int)(id % npw);
    const c2<T> v = box[(int64_t)b * boxsz + pos[q]];
    dC[id].x += (double)v.x;
    dC[id].y += (double)v.y;
  }
}

template <typename T>
cudaError_t launch_gather_box(const c2<T>* box, int nb, int npw, const int* pos, int64_t boxsz, double2* dC,
                              cudaStream_t s) {
  const int64_t total = (int64_t)nb * npw;
  if (total == 0) return cudaSuccess;
  gather_box_kernel<T><<<gridx(total), 256, 0, s>>>(box, nb, npw, pos, boxsz, dC);
  return cudaGetLastError();
}

#define RPA_ADJ_INST(T)                                                                                                \
  template cudaError_t launch_nbar<T>(const c2<T>*, int64_t, int, const T*, const c2<T>*, int, c2<T>*, cudaStream_t);  \
  template cudaError_t launch_paw_adjoint<T>(const c2<T>*, const c2<T>*, const c2<T>*, int, int, int, int,             \
                                             const double2*, const int*, const int*, const int*, const int64_t*,       \
                                             const int*, const int*, const int*, c2<T>*, double2*, double2*, double2*, \
                                             cudaStream_t);                                                            \
  template cudaError_t launch_adj_stageC<T>(const c2<T>*, int, int64_t, int, int, int, int, int, const int*,          \
                                            const int*, const int*, double, const c2<T>*, c2<T>*, cudaStream_t);       \
  template size_t adj_stageA_fused_smem<T>(int, int, int);                                                             \
  template cudaError_t launch_adj_stageA_fused<T>(const c2<T>*, int, int, int, int, int, const c2<T>*, const c2<T>*,   \
                                                  const c2<T>*, const c2<T>*, const int*, int, c2<T>*, c2<T>*, c2<T>*, \
                                                  c2<T>*, cudaStream_t);                                               \
  template cudaError_t launch_adj_stageA<T>(const c2<T>*, int, int, int, int, const c2<T>*, const c2<T>*,              \
                                            const c2<T>*, const int*, int, int64_t, c2<T>*, c2<T>*, cudaStream_t);     \
  template cudaError_t launch_adj_un<T>(const c2<T>*, int, int64_t, const c2<T>*, const int*, int, int64_t, c2<T>*,    \
                                        cudaStream_t);                                                                 \
  template cudaError_t launch_twiddle_adj<T>(c2<T>*, int, int, int, int, cudaStream_t);                                \
  template cudaError_t launch_gather_box<T>(const c2<T>*, int, int, const int*, int64_t, double2*, cudaStream_t);

RPA_ADJ_INST(float)
RPA_ADJ_INST(double)

}  // namespace rpa
