// FP64 log-determinant of 1 - v^1/2 chi0 v^1/2 for the RPA correlation
// energy (Eqs. 1-2; Table 1 step 13), batched over frequencies.
//
// chi0 <= 0 makes A = 1 - M Hermitian positive definite with eigenvalues
// >= 1, so a Cholesky factorisation A = L L^H needs no pivoting and
// ln det A = sum_i ln(L_ii^2).  The blocked right-looking factorisation uses
// 32-wide panels: the diagonal block is factorised by one CTA per frequency,
// the panel below it by a triangular solve, and the trailing lower triangle is
// updated with 64x64 DFMA tiles.  A pivot that is not positive (or NaN) sets a
// device flag that the host turns into RPA_ERR_NOT_HPD; the kernels never trap.
//
// In the mixed-precision modes the part of the matrix that is still being
// updated is held in float-float form (each real value the unevaluated sum of
// two FP32 numbers, about 48 significant bits) and the trailing updates run on
// the FP32 pipe; GB300's FP64 pipe retires only a few lanes per clock, so even
// format conversions there would cost as much as the updates.  Factorised
// columns are written back in FP64, so the finished factor has one format.
#include "ff_math.cuh"
#include "rpa.h"
#include <algorithm>

#include "rpa_internal.h"

namespace rpa {

constexpr int CB = 32;  // panel width
constexpr int UT = 64;  // update tile edge

// A = 1 - v^1/2 chi v^1/2 (lower triangle), in FP64 or float-float (FF).
template <bool FF>
__global__ void chol_form_kernel(const double2* __restrict__ chi, const double* __restrict__ v, int nw, int NG,
                                 double2* __restrict__ A) {
  const int64_t total = (int64_t)nw * NG * NG;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(id % NG);
    const int64_t r = id / NG;
    const int i = (int)(r % NG);
    if (j > i) continue;
    const double s = sqrt(v[i]) * sqrt(v[j]);
    const double2 c = chi[id];
    double2 a = make_double2(-s * c.x, -s * c.y);
    if (i == j) {
      a.x += 1.0;
      a.y = 0.0;
    }
    if constexpr (FF) reinterpret_cast<float4*>(A)[id] = ff_split(a); else A[id] = a;
  }
}

__global__ void trace_kernel(const double2* __restrict__ chi, const double* __restrict__ v, int NG,
                             double* __restrict__ trace) {
  __shared__ double red[256];
  const int w = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < NG; i += blockDim.x) s += v[i] * chi[((int64_t)w * NG + i) * NG + i].x;
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) trace[w] = red[0];
}

// 1/sqrt(x) for a pivot x > 0: a single-precision estimate refined by two
// Newton steps y <- y (3 - x y^2) / 2 in FP64 (quadratic convergence from
// about 2^-22 to full precision).  One short dependent chain replaces a square
// root followed by a division on the serial path of the panel factorisation.
__device__ __forceinline__ double rsqrt_newton(double x) {
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);
  double y = (double)rsqrtf((float)x);
  const double hx = 0.5 * x;
  y = y * fma(-hx, y * y, 1.5);
  y = y * fma(-hx, y * y, 1.5);
  return y;
}

// One CTA per frequency factorises the b x b diagonal block in place, adds
// the logs of its pivots to logdet[w] (ln det A = sum_i ln L_ii^2) and writes
// the inverse of the factor to Linv[w] (CB x CB, lower triangle, zero above).
// Every column step is parallel over the CTA: the column of L is scaled, then
// the Schur complement and the forward substitution for L^-1 (right-hand side
// I) are updated together; the logs are taken once at the end.
// FF: the block is read in float-float form and the inverse is also written
// in float-float form to Linv_ff; the factor always goes back in FP64.
// Body for one matrix Aw (its logdet slot, flag and CB x CB inverse slices).
template <bool FF>
__device__ __forceinline__ void chol_diag_body(double2* __restrict__ Aw, int NG, int k0, int b, double* ld_w,
                                               int* __restrict__ flag, double2* __restrict__ Lw,
                                               float4* __restrict__ Lffw) {
  __shared__ double2 L[CB][CB + 1];
  __shared__ double2 X[CB][CB + 1];  // right-hand side I, then L^-1
  __shared__ double piv_s[CB];
  __shared__ double dinv_s;
  const int tid = threadIdx.x;
  for (int e = tid; e < CB * CB; e += blockDim.x) {
    const int i = e / CB, j = e % CB;
    double2 a = make_double2(0.0, 0.0);
    if (i < b && j <= i) {
      const int64_t o = (int64_t)(k0 + i) * NG + k0 + j;
      if constexpr (FF) a = ff_to_double(reinterpret_cast<const float4*>(Aw)[o]); else a = Aw[o];
    }
    L[i][j] = a;
    X[i][j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int c = 0; c < b; ++c) {
    // one thread takes the pivot (the FP64 pipe retires only a few lanes per
    // clock, so the other threads must not repeat the square root)
    if (tid == 0) {
      double piv = L[c][c].x;
      if (!(piv > 0.0)) {
        atomicExch(flag, 1);
        piv = 1.0;
      }
      piv_s[c] = piv;
      dinv_s = rsqrt_newton(piv);
    }
    __syncthreads();
    const double dinv = dinv_s, piv = piv_s[c];
    if (tid < CB) {
      if (tid > c && tid < b) {
        L[tid][c].x *= dinv;
        L[tid][c].y *= dinv;
      } else if (tid == c) {
        L[c][c] = make_double2(piv * dinv, 0.0);
      }
    } else if (tid < 2 * CB && tid - CB <= c) {
      X[c][tid - CB].x *= dinv;
      X[c][tid - CB].y *= dinv;
    }
    __syncthreads();
    // The FP64 pipe retires a warp instruction in many cycles whatever its
    // active lanes, so the useful elements are enumerated densely: first the
    // Schur complement triangle (c < j <= i < b), then the m x (c+1) block of
    // the forward substitution.
    const int m = b - c - 1;
    const int ntri = m * (m + 1) / 2;
    for (int e = tid; e < ntri + m * (c + 1); e += blockDim.x) {
      if (e < ntri) {
        int r = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
        while (r * (r + 1) / 2 > e) --r;
        while ((r + 1) * (r + 2) / 2 <= e) ++r;
        const int i = c + 1 + r, j = c + 1 + (e - r * (r + 1) / 2);
        // Schur complement: L_ij -= L_ic conj(L_jc)
        const double2 x = L[i][c], y = L[j][c];
        L[i][j].x -= x.x * y.x + x.y * y.y;
        L[i][j].y -= x.y * y.x - x.x * y.y;
      } else {
        const int f = e - ntri;
        const int i = c + 1 + f / (c + 1), j = f % (c + 1);
        // forward substitution: X_ij -= L_ic X_cj
        const double2 x = L[i][c], y = X[c][j];
        X[i][j].x -= x.x * y.x - x.y * y.y;
        X[i][j].y -= x.x * y.y + x.y * y.x;
      }
    }
    __syncthreads();
  }
  if (tid < 32) {
    double ld = tid < b ? log(piv_s[tid]) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ld += __shfl_xor_sync(0xffffffffu, ld, o);
    if (tid == 0) *ld_w += ld;
  }
  for (int e = tid; e < CB * CB; e += blockDim.x) {
    const int i = e / CB, j = e % CB;
    const double2 x = (i < b && j <= i) ? X[i][j] : make_double2(0.0, 0.0);
    Lw[e] = x;
    if constexpr (FF) Lffw[e] = ff_split(x);
    if (i < b && j <= i) Aw[(int64_t)(k0 + i) * NG + k0 + j] = L[i][j];
  }
}

template <bool FF>
__global__ void __launch_bounds__(256) chol_diag_kernel(double2* __restrict__ A, int NG, int k0, int b,
                                                        double* __restrict__ logdet, int* __restrict__ flag,
                                                        double2* __restrict__ Linv, float4* __restrict__ Linv_ff) {
  const int w = blockIdx.x;
  chol_diag_body<FF>(A + (int64_t)w * NG * NG, NG, k0, b, logdet + w, flag, Linv + (int64_t)w * CB * CB,
                     FF ? Linv_ff + (int64_t)w * CB * CB : nullptr);
}

// Panel below the diagonal block: X = A_panel L_kk^-H, i.e.
// x_rj = sum_{l <= j} a_rl conj(Linv_jl).  16 threads per row, each owning
// columns j and b-1-j so that every thread does b+1 multiply-adds.  FF: the
// panel rows and the inverse are read in float-float form, the product is
// float-float, and the result goes to A in FP64 and to Lp ([NG][CB] per
// frequency, float-float) for the trailing update.
constexpr int TROWS = 16;  // rows per triangular-solve CTA

// Body for one matrix Aw, its inverse slices and its panel Pw ([NG][CB]), row tile bx.
template <bool FF>
__device__ __forceinline__ void chol_trsm_body(double2* __restrict__ Aw, int NG, int k0, int b,
                                               const double2* __restrict__ Lw, const float4* __restrict__ Lffw,
                                               float4* __restrict__ Pw, int bx) {
  using E = typename std::conditional<FF, float4, double2>::type;
  __shared__ E Li[CB][CB + 1];
  __shared__ E X[TROWS][CB + 1];
  const int i0 = k0 + b + bx * TROWS;
  for (int e = threadIdx.x; e < CB * CB; e += blockDim.x) {
    if constexpr (FF) Li[e / CB][e % CB] = Lffw[e];
    else Li[e / CB][e % CB] = Lw[e];
  }
  for (int e = threadIdx.x; e < TROWS * CB; e += blockDim.x) {
    const int r = e / CB, l = e % CB;
    const bool in = i0 + r < NG && l < b;
    const int64_t o = (int64_t)(i0 + r) * NG + k0 + l;
    if constexpr (FF) X[r][l] = in ? reinterpret_cast<const float4*>(Aw)[o] : make_float4(0.f, 0.f, 0.f, 0.f);
    else X[r][l] = in ? Aw[o] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int r = threadIdx.x >> 4, t = threadIdx.x & 15;
  const int row = i0 + r;
  if (row >= NG) return;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    // t owns column t when t <= b-1-t, and column b-1-t when that lies above t
    const int j = h == 0 ? t : b - 1 - t;
    if (h == 0 ? 2 * t > b - 1 : j <= t) continue;
    if constexpr (FF) {
      float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int l = 0; l <= j; ++l) {
        const float4 a = X[r][l], y = Li[j][l];
        ff_mac(s.x, s.y, a.x, a.y, y.x, y.y);
        ff_mac(s.x, s.y, a.z, a.w, y.z, y.w);
        ff_mac(s.z, s.w, a.z, a.w, y.x, y.y);
        ff_mac(s.z, s.w, -a.x, -a.y, y.z, y.w);
      }
      ff_norm(s.x, s.y);
      ff_norm(s.z, s.w);
      Aw[(int64_t)row * NG + k0 + j] = ff_to_double(s);
      Pw[(int64_t)row * CB + j] = s;
    } else {
      double2 s = make_double2(0.0, 0.0);
      for (int l = 0; l <= j; ++l) cmac_cj<double>(s, X[r][l], Li[j][l]);
      Aw[(int64_t)row * NG + k0 + j] = s;
    }
  }
}

template <bool FF>
__global__ void __launch_bounds__(256) chol_trsm_kernel(double2* __restrict__ A, int NG, int k0, int b,
                                                        const double2* __restrict__ Linv,
                                                        const float4* __restrict__ Linv_ff, float4* __restrict__ Lp) {
  const int w = blockIdx.y;
  chol_trsm_body<FF>(A + (int64_t)w * NG * NG, NG, k0, b, Linv + (int64_t)w * CB * CB,
                     FF ? Linv_ff + (int64_t)w * CB * CB : nullptr, FF ? Lp + (int64_t)w * NG * CB : nullptr,
                     blockIdx.x);
}

__device__ __forceinline__ void tri_tile(int t, int& ti, int& tj) {
  int i = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (i * (i + 1) / 2 > t) --i;
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  ti = i;
  tj = t - i * (i + 1) / 2;
}

__global__ void __launch_bounds__(256) chol_update_kernel(double2* __restrict__ A, int NG, int k0, int b) {
  extern __shared__ double2 upd_smem[];
  double2 (*Li)[UT] = reinterpret_cast<double2 (*)[UT]>(upd_smem);
  double2 (*Lj)[UT] = reinterpret_cast<double2 (*)[UT]>(upd_smem + CB * UT);
  const int w = blockIdx.y;
  double2* Aw = A + (int64_t)w * NG * NG;
  int ti, tj;
  tri_tile(blockIdx.x, ti, tj);
  const int s0 = k0 + b;
  const int r0 = s0 + ti * UT, c0 = s0 + tj * UT;
  for (int e = threadIdx.x; e < b * UT; e += blockDim.x) {
    const int rr = e / b, l = e % b;
    Li[l][rr] = (r0 + rr < NG) ? Aw[(int64_t)(r0 + rr) * NG + k0 + l] : make_double2(0.0, 0.0);
    Lj[l][rr] = (c0 + rr < NG) ? Aw[(int64_t)(c0 + rr) * NG + k0 + l] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double2 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_double2(0.0, 0.0);
  for (int l = 0; l < b; ++l) {
    double2 a[4], bb[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) a[r] = Li[l][ty + 16 * r];
#pragma unroll
    for (int c = 0; c < 4; ++c) bb[c] = Lj[l][tx + 16 * c];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) cmac_cj<double>(acc[r][c], a[r], bb[c]);
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int row = r0 + ty + 16 * r, col = c0 + tx + 16 * c;
      if (row < NG && col < NG && col <= row) {
        double2* p = Aw + (int64_t)row * NG + col;
        double2 v = *p;
        v.x -= acc[r][c].x;
        v.y -= acc[r][c].y;
        *p = v;
      }
    }
}

// Float-float trailing update on 32 x 32 tiles of 64 threads (4 x 4 outputs
// each): the panel comes from Lp and the trailing matrix is float-float, so
// the kernel issues no FP64 instruction.  The accumulators take 167 registers
// a thread; small CTAs let six of them share an SM so that twelve warps hide
// the latency of the dependent two-sum steps.  The tiles cover the lower
// triangle of the square from row/column s0 to NG, or with strip set only its
// first 32-column strip (which is the next panel, as UTF == CB).
constexpr int UTF = 32;
static_assert(UTF == CB, "the look-ahead strip of the trailing update is one panel wide");

// Body for one matrix (A_w in float-float form) and its panel Pw, tile (ti, tj) from s0.
__device__ __forceinline__ void chol_update_ff_body(double2* __restrict__ A_w, int NG, int k0, int b, int s0, int ti,
                                                    int tj, const float4* __restrict__ Pw) {
  __shared__ float4 Li[CB][UTF];
  __shared__ float4 Lj[CB][UTF];
  float4* Aw = reinterpret_cast<float4*>(A_w);
  const int r0 = s0 + ti * UTF, c0 = s0 + tj * UTF;
  for (int e = threadIdx.x; e < b * UTF; e += blockDim.x) {
    const int rr = e / b, l = e % b;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    Li[l][rr] = (r0 + rr < NG) ? Pw[(int64_t)(r0 + rr) * CB + l] : z;
    Lj[l][rr] = (c0 + rr < NG) ? Pw[(int64_t)(c0 + rr) * CB + l] : z;
  }
  __syncthreads();
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  // acc[r][c] = (re hi, re lo, im hi, im lo) of sum_l L_il conj(L_jl)
  float4 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
  for (int l = 0; l < b; ++l) {
    float4 y[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) y[c] = Lj[l][tx + 8 * c];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float4 a = Li[l][ty + 8 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float4& s = acc[r][c];
        // a * conj(y): re = ar yr + ai yi, im = ai yr - ar yi
        ff_mac(s.x, s.y, a.x, a.y, y[c].x, y[c].y);
        ff_mac(s.x, s.y, a.z, a.w, y[c].z, y[c].w);
        ff_mac(s.z, s.w, a.z, a.w, y[c].x, y[c].y);
        ff_mac(s.z, s.w, -a.x, -a.y, y[c].z, y[c].w);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int row = r0 + ty + 8 * r, col = c0 + tx + 8 * c;
      if (row < NG && col < NG && col <= row) {
        float4* p = Aw + (int64_t)row * NG + col;
        float4 v = *p;
        ff_sub(v.x, v.y, acc[r][c].x, acc[r][c].y);
        ff_sub(v.z, v.w, acc[r][c].z, acc[r][c].w);
        *p = v;
      }
    }
}

__global__ void __launch_bounds__(64, 6) chol_update_ff_kernel(double2* __restrict__ A, int NG, int k0, int b, int s0,
                                                               int strip, const float4* __restrict__ Lp) {
  const int w = blockIdx.y;
  int ti = blockIdx.x, tj = 0;
  if (!strip) tri_tile(blockIdx.x, ti, tj);
  // A holds 16-byte elements (double2, or float4 in float-float form)
  chol_update_ff_body(A + (int64_t)w * NG * NG, NG, k0, b, s0, ti, tj, Lp + (int64_t)w * NG * CB);
}

__global__ void add_terms_kernel(const double* __restrict__ ld, const double* __restrict__ tr, int nw,
                                 double* __restrict__ terms) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w < nw) terms[w] = ld[w] + tr[w];
}

static inline int gridc(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b > 152 * 64 ? 152 * 64 : (b < 1 ? 1 : b));
}

// work layout (complex slots of 16 bytes): the matrix [nw][NG][NG], the
// inverses of the diagonal blocks in FP64 and in float-float [nw][CB][CB]
// each, and two float-float panels [nw][NG][CB] (alternate panels, so that the
// look-ahead can solve panel k+1 while the update of panel k still reads its own)
int64_t logdet_work_elems(int nw, int NG) {
  return (int64_t)nw * NG * NG + 2 * (int64_t)nw * CB * CB + 2 * (int64_t)nw * NG * CB;
}

// Launch on stream s with the given scheduling priority (lower is more urgent),
// so that the short kernels of the look-ahead chain take SMs as soon as
// trailing-update CTAs retire; the attribute also holds in a captured graph.
template <typename... KArgs, typename... Args>
static cudaError_t launch_prio(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, int prio,
                               Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributePriority;
  at[0].val.priority = prio;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Float-float factorisation with a look-ahead of one panel.  The update of
// panel k is split into its first column strip (panel k+1, on s, high
// priority) and the rest (on the second stream).  Panel k+1 is factorised and
// solved on s while the rest of the update of panel k runs beside it; the
// strip update of panel k+1 waits for that rest, which also wrote the strip.
// Events: ev_t (panel solved, s -> s2) and ev_u (rest updated, s2 -> s); s
// waits for the last rest at the end, so the sequence can be captured.
static cudaError_t run_logdet_ff_lookahead(int nw, int NG, double2* work, double* logdet, int* flag,
                                           const LogdetStreams& la, cudaStream_t s, int64_t* nl) {
  cudaError_t e;
  int least = 0, greatest = 0;
  if ((e = cudaDeviceGetStreamPriorityRange(&least, &greatest)) != cudaSuccess) return e;
  double2* Linv = work + (int64_t)nw * NG * NG;
  float4* Linv_ff = reinterpret_cast<float4*>(Linv + (int64_t)nw * CB * CB);
  float4* Lp0 = Linv_ff + (int64_t)nw * CB * CB;
  bool rest_pending = false;  // a rest update has been issued on s2 and not yet waited for by s
  for (int k0 = 0, k = 0; k0 < NG; k0 += CB, ++k) {
    const int b = (NG - k0) < CB ? (NG - k0) : CB;
    const int rest = NG - k0 - b;
    float4* Lp = Lp0 + (int64_t)(k & 1) * nw * NG * CB;
    if ((e = launch_prio(chol_diag_kernel<true>, dim3(nw), dim3(256), s, greatest, work, NG, k0, b, logdet, flag,
                         Linv, Linv_ff)) != cudaSuccess)
      return e;
    ++*nl;
    if (rest == 0) break;
    const dim3 tg((rest + TROWS - 1) / TROWS, nw);
    if ((e = launch_prio(chol_trsm_kernel<true>, tg, dim3(256), s, greatest, work, NG, k0, b,
                         (const double2*)Linv, (const float4*)Linv_ff, Lp)) != cudaSuccess)
      return e;
    ++*nl;
    const int nt = (rest + UTF - 1) / UTF;
    const int s0 = k0 + b;
    if (nt > 1) {
      if ((e = cudaEventRecord(la.ev_t, s)) != cudaSuccess) return e;
    }
    // the strip (next panel) was last written by the rest update of panel k-1
    if (rest_pending) {
      if ((e = cudaStreamWaitEvent(s, la.ev_u, 0)) != cudaSuccess) return e;
      rest_pending = false;
    }
    if ((e = launch_prio(chol_update_ff_kernel, dim3(nt, nw), dim3(64), s, greatest, work, NG, k0, b, s0, 1,
                         (const float4*)Lp)) != cudaSuccess)
      return e;
    ++*nl;
    if (nt > 1) {
      const int nr = nt - 1;
      if ((e = cudaStreamWaitEvent(la.s2, la.ev_t, 0)) != cudaSuccess) return e;
      chol_update_ff_kernel<<<dim3(nr * (nr + 1) / 2, nw), 64, 0, la.s2>>>(work, NG, k0, b, s0 + UTF, 0, Lp);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = cudaEventRecord(la.ev_u, la.s2)) != cudaSuccess) return e;
      rest_pending = true;
      ++*nl;
    }
  }
  if (rest_pending) {
    if ((e = cudaStreamWaitEvent(s, la.ev_u, 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t run_logdet(const double2* chi, const double* v, int nw, int NG, double2* work, double* logdet,
                       double* trace, int* flag, bool ff_update, cudaStream_t s, int64_t* launches,
                       const LogdetStreams* la, cudaEvent_t formed) {
  cudaError_t e;
  int64_t nl = 0;
  const int upd_smem = 2 * CB * UT * (int)sizeof(double2);
  if ((e = cudaFuncSetAttribute(chol_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, upd_smem)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(logdet, 0, sizeof(double) * nw, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(flag, 0, sizeof(int), s)) != cudaSuccess) return e;
  double2* Linv = work + (int64_t)nw * NG * NG;                                     // [nw][CB][CB]
  float4* Linv_ff = reinterpret_cast<float4*>(Linv + (int64_t)nw * CB * CB);        // [nw][CB][CB]
  float4* Lp = Linv_ff + (int64_t)nw * CB * CB;                                     // [nw][NG][CB]
  const int64_t total = (int64_t)nw * NG * NG;
  if (ff_update)
    chol_form_kernel<true><<<gridc(total), 256, 0, s>>>(chi, v, nw, NG, work);
  else
    chol_form_kernel<false><<<gridc(total), 256, 0, s>>>(chi, v, nw, NG, work);
  trace_kernel<<<nw, 256, 0, s>>>(chi, v, NG, trace);
  nl += 2;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (formed && (e = cudaEventRecord(formed, s)) != cudaSuccess) return e;
  if (ff_update && la) {
    e = run_logdet_ff_lookahead(nw, NG, work, logdet, flag, *la, s, &nl);
    if (launches) *launches += nl;
    return e;
  }
  for (int k0 = 0; k0 < NG; k0 += CB) {
    const int b = (NG - k0) < CB ? (NG - k0) : CB;
    const int rest = NG - k0 - b;
    const dim3 tg((rest + TROWS - 1) / TROWS, nw);
    if (ff_update) {
      chol_diag_kernel<true><<<nw, 256, 0, s>>>(work, NG, k0, b, logdet, flag, Linv, Linv_ff);
      if (rest > 0) {
        chol_trsm_kernel<true><<<tg, 256, 0, s>>>(work, NG, k0, b, Linv, Linv_ff, Lp);
        const int nt = (rest + UTF - 1) / UTF;
        chol_update_ff_kernel<<<dim3(nt * (nt + 1) / 2, nw), 64, 0, s>>>(work, NG, k0, b, k0 + b, 0, Lp);
      }
    } else {
      chol_diag_kernel<false><<<nw, 256, 0, s>>>(work, NG, k0, b, logdet, flag, Linv, nullptr);
      if (rest > 0) {
        chol_trsm_kernel<false><<<tg, 256, 0, s>>>(work, NG, k0, b, Linv, nullptr, nullptr);
        const int nt = (rest + UT - 1) / UT;
        chol_update_kernel<<<dim3(nt * (nt + 1) / 2, nw), 256, upd_smem, s>>>(work, NG, k0, b);
      }
    }
    nl += rest > 0 ? 3 : 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (launches) *launches += nl;
  return cudaSuccess;
}

// ---------------------------------------------------------------- batched log-det
// The float-float factorisation (one stream, no look-ahead) of many matrices of
// different orders in one set of launches: matrix m of the batch is one
// frequency of one instance, described by LdMat (its own work slices and
// outputs).  Every launch covers all matrices; a CTA whose matrix is already
// factorised, or whose tile lies outside it, returns at once.  Per matrix the
// arithmetic and its order are those of run_logdet with the float-float
// update (bit-identical).
__global__ void chol_form_batch_kernel(const LdMat* __restrict__ d) {
  const LdMat m = d[blockIdx.y];
  const int64_t total = (int64_t)m.NG * m.NG;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *m.logdet = 0.0;
    *m.flag = 0;  // every matrix of the instance writes 0 before any pivot is taken
  }
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(id % m.NG), i = (int)(id / m.NG);
    if (j > i) continue;
    const double sc = sqrt(m.v[i]) * sqrt(m.v[j]);
    const double2 c = m.chi[id];
    double2 a = make_double2(-sc * c.x, -sc * c.y);
    if (i == j) {
      a.x += 1.0;
      a.y = 0.0;
    }
    reinterpret_cast<float4*>(m.A)[id] = ff_split(a);
  }
}

__global__ void trace_batch_kernel(const LdMat* __restrict__ d) {
  __shared__ double red[256];
  const LdMat m = d[blockIdx.x];
  double s = 0.0;
  for (int i = threadIdx.x; i < m.NG; i += blockDim.x) s += m.v[i] * m.chi[(int64_t)i * m.NG + i].x;
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *m.trace = red[0];
}

__global__ void __launch_bounds__(256) chol_diag_batch_kernel(const LdMat* __restrict__ d, int k0) {
  const LdMat m = d[blockIdx.x];
  if (k0 >= m.NG) return;
  chol_diag_body<true>(m.A, m.NG, k0, min(CB, m.NG - k0), m.logdet, m.flag, m.Linv, m.Linv_ff);
}

__global__ void __launch_bounds__(256) chol_trsm_batch_kernel(const LdMat* __restrict__ d, int k0) {
  const LdMat m = d[blockIdx.y];
  const int b = min(CB, m.NG - k0);
  if (k0 + b >= m.NG || k0 + b + (int)blockIdx.x * TROWS >= m.NG) return;
  chol_trsm_body<true>(m.A, m.NG, k0, b, m.Linv, m.Linv_ff, m.Lp, blockIdx.x);
}

__global__ void __launch_bounds__(64, 6) chol_update_ff_batch_kernel(const LdMat* __restrict__ d, int k0) {
  const LdMat m = d[blockIdx.y];
  const int b = min(CB, m.NG - k0);
  const int rest = m.NG - k0 - b;
  if (rest <= 0) return;
  const int nt = (rest + UTF - 1) / UTF;
  if ((int)blockIdx.x >= nt * (nt + 1) / 2) return;
  int ti, tj;
  tri_tile(blockIdx.x, ti, tj);
  chol_update_ff_body(m.A, m.NG, k0, b, k0 + b, ti, tj, m.Lp);
}

// The slices of run_logdet's work buffer for frequency w (matrix, inverses, first panel).
LdMat logdet_mat(double2* work, int nw, int NG, int w) {
  LdMat m{};
  double2* Linv = work + (int64_t)nw * NG * NG;
  float4* Lff = reinterpret_cast<float4*>(Linv + (int64_t)nw * CB * CB);
  float4* Lp = Lff + (int64_t)nw * CB * CB;
  m.A = work + (int64_t)w * NG * NG;
  m.Linv = Linv + (int64_t)w * CB * CB;
  m.Linv_ff = Lff + (int64_t)w * CB * CB;
  m.Lp = Lp + (int64_t)w * NG * CB;
  m.NG = NG;
  return m;
}

cudaError_t run_logdet_batch(const LdMat* d, int nmat, int maxNG, cudaStream_t s, int64_t* launches) {
  if (nmat == 0 || maxNG == 0) return cudaSuccess;
  int64_t nl = 0;
  const int fx = (int)std::min<int64_t>(((int64_t)maxNG * maxNG + 255) / 256, 64);
  chol_form_batch_kernel<<<dim3(fx, nmat), 256, 0, s>>>(d);
  trace_batch_kernel<<<nmat, 256, 0, s>>>(d);
  nl += 2;
  cudaError_t e;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int k0 = 0; k0 < maxNG; k0 += CB) {
    const int b = std::min(CB, maxNG - k0);
    const int rest = maxNG - k0 - b;
    chol_diag_batch_kernel<<<nmat, 256, 0, s>>>(d, k0);
    ++nl;
    if (rest > 0) {
      chol_trsm_batch_kernel<<<dim3((rest + TROWS - 1) / TROWS, nmat), 256, 0, s>>>(d, k0);
      const int nt = (rest + UTF - 1) / UTF;
      chol_update_ff_batch_kernel<<<dim3(nt * (nt + 1) / 2, nmat), 64, 0, s>>>(d, k0);
      nl += 2;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (launches) *launches += nl;
  return cudaSuccess;
}

// ---------------------------------------------------------------- allocation-free entry point
// Scratch of rpa_logdet_noalloc: the Cholesky work matrix (up to
// kNoAllocMaxElems complex elements), the inverses of the diagonal blocks (CB^2
// per frequency), the per-frequency log-det and trace accumulators and the
// pivot flag.  It lives for the life of the process on every device that loads
// the library (17 MiB + 1040 B).
constexpr int64_t kNoAllocMaxElems = (int64_t)1 << 20;
constexpr int kNoAllocMaxNw = 64;
constexpr int64_t kNoAllocLinv = (int64_t)kNoAllocMaxNw * CB * CB;
constexpr int64_t kNoAllocSlots = kNoAllocMaxElems + kNoAllocLinv + kNoAllocMaxNw + 1;  // double2 slots
static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocSlots];

}  // namespace rpa

#include <mutex>

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kMaxDevices] = {nullptr};
}  // namespace

extern "C" rpa_status rpa_logdet_noalloc(const double* chi, const double* v, int32_t nw, int32_t ng, double* terms,
                                         void* stream) {
  using namespace rpa;
  if (!chi || !v || !terms || nw < 1 || ng < 1) return RPA_ERR_ARG;
  if (nw > kNoAllocMaxNw || (int64_t)nw * ng * ng > kNoAllocMaxElems) return RPA_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return RPA_ERR_CUDA;
  }
  for (const void* p : {(const void*)chi, (const void*)v, (const void*)terms}) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      return RPA_ERR_ARG;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return RPA_ERR_ARG;
    // device memory of another GPU is not readable by this device's kernels
    if (a.type == cudaMemoryTypeDevice && a.device != dev) return RPA_ERR_ARG;
  }
  // one-time set-up per device: the device address of the static scratch
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return RPA_ERR_CUDA;
      }
      g_noalloc_addr[dev] = p;
    }
    base = g_noalloc_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  double2* work = (double2*)base;
  double* ld = (double*)(work + kNoAllocMaxElems + kNoAllocLinv);  // past the matrix and the block inverses
  double* tr = ld + kNoAllocMaxNw;
  int* flag = (int*)(tr + kNoAllocMaxNw);
  // run_logdet clears the log-det accumulators and the flag itself; the work
  // matrix is fully rewritten from chi before it is read
  if (run_logdet((const double2*)chi, v, nw, ng, work, ld, tr, flag, false, s, nullptr) != cudaSuccess) return RPA_ERR_CUDA;
  add_terms_kernel<<<(nw + 63) / 64, 64, 0, s>>>(ld, tr, nw, terms);
  if (cudaGetLastError() != cudaSuccess) return RPA_ERR_CUDA;
  int h_flag = 0;
  if (cudaMemcpyAsync(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return RPA_ERR_CUDA;
  }
  return h_flag ? RPA_ERR_NOT_HPD : RPA_OK;
}
