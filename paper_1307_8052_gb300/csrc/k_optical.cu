// Optical limit q -> 0 (Eqs. 12-14): the G = 0 pair density of a q = 0 point
// per unit |q| along q^,
//   n_nm(0) = -i q^.<psi_n|grad|psi_m> / (e_m - e_n),
//   q^.<psi_n|grad|psi_m> = i sum_Q conj(C_n(Q)) q^.(k+Q) C_m(Q)
//                           + sum_ij conj(P_ni) (q^.Q_grad)_ij P_mj,
// written into the G = 0 column of a block of pair densities.  The plane-wave
// part is exact in the basis (the spectral gradient); q^.Q_grad (Eq. 14) is an
// input contracted with q^ on the host.  FP64 throughout: the head enters the
// log-det with the largest Coulomb weight.
#include "rpa.h"
#include "rpa_internal.h"

#include <algorithm>

namespace rpa {

constexpr int OT = 64;  // output tile edge along the empty bands (pairs)
constexpr int OK = 16;  // K chunk

// Y[b][i] = sum_j Qn[i][j] P[R[b]][j]
__global__ void optical_paw_y_kernel(const double2* __restrict__ P, int KP, const double2* __restrict__ Qn,
                                     const int* __restrict__ R, int nR, double2* __restrict__ Y) {
  const int64_t total = (int64_t)nR * KP;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(id % KP);
    const int b = (int)(id / KP);
    const double2* pm = P + (int64_t)R[b] * KP;
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < KP; ++j) cmac<double>(acc, Qn[(int64_t)i * KP + j], pm[j]);
    Y[id] = acc;
  }
}

// Partial D[a][b] = sum_k A_k(n_a) B_k(m_b) over this CTA's slice of K = npw
// (+ KP), RT x 4 outputs a thread on a (16 RT) x 64 tile, into
// Dp[split][nL][nR].  The row tile follows nL (the occupied bands of a block,
// often 16 or fewer) so that no FP64 work goes to padding rows; the K
// dimension is split across CTAs because the tile count is small.  Global
// reads run along K (16 consecutive coefficients of one band per 16 threads);
// the shared tiles are padded by one element against bank conflicts.
template <typename T, int RT>
__global__ void __launch_bounds__(256) optical_dipole_kernel(const double2* __restrict__ C, int npw,
                                                             const double* __restrict__ s,
                                                             const double2* __restrict__ P, int KP,
                                                             const double2* __restrict__ Y,
                                                             const int* __restrict__ L, int nL,
                                                             const int* __restrict__ R, int nR, int kslice,
                                                             double2* __restrict__ Dp) {
  constexpr int TL = 16 * RT;
  __shared__ double2 As[OK][TL + 1];
  __shared__ double2 Bs[OK][OT + 1];
  const int a0 = blockIdx.y * TL, b0 = blockIdx.x * OT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double2 acc[RT][4];
#pragma unroll
  for (int r = 0; r < RT; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_double2(0.0, 0.0);
  const int K = npw + (P ? KP : 0);
  const int kbeg = blockIdx.z * kslice, kend = min(K, kbeg + kslice);
  const int kk = threadIdx.x % OK, rr = threadIdx.x / OK;  // 16 rows x 16 k per pass
  for (int k0 = kbeg; k0 < kend; k0 += OK) {
    const int k = k0 + kk;
#pragma unroll
    for (int q = 0; q < RT; ++q) {
      const int r = rr + 16 * q;
      double2 av = make_double2(0.0, 0.0);
      if (k < kend && a0 + r < nL) {
        const int n = L[a0 + r];
        if (k < npw) {
          // i s(Q) conj(C_n(Q))
          const double2 cn = C[(int64_t)n * npw + k];
          av = make_double2(s[k] * cn.y, s[k] * cn.x);
        } else {
          const double2 pn = P[(int64_t)n * KP + (k - npw)];
          av = make_double2(pn.x, -pn.y);
        }
      }
      As[kk][r] = av;
    }
#pragma unroll
    for (int q = 0; q < OT / 16; ++q) {
      const int r = rr + 16 * q;
      double2 bv = make_double2(0.0, 0.0);
      if (k < kend && b0 + r < nR) {
        const int m = R[b0 + r];
        bv = k < npw ? C[(int64_t)m * npw + k] : Y[(int64_t)(b0 + r) * KP + (k - npw)];
      }
      Bs[kk][r] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < OK; ++j) {
      double2 av[RT], bv[4];
#pragma unroll
      for (int r = 0; r < RT; ++r) av[r] = As[j][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Bs[j][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < RT; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) cmac<double>(acc[r][c], av[r], bv[c]);
    }
    __syncthreads();
  }
  double2* Dz = Dp + (int64_t)blockIdx.z * nL * nR;
#pragma unroll
  for (int r = 0; r < RT; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int a = a0 + ty + 16 * r, b = b0 + tx + 16 * c;
      if (a < nL && b < nR) Dz[(int64_t)a * nR + b] = acc[r][c];
    }
}

// N[(a nR + b) NG + ig0] = -i D / (e_m - e_n), D the sum of the nsplit partials
template <typename T>
__global__ void optical_head_kernel(const double2* __restrict__ Dp, int nsplit, const int* __restrict__ L, int nL,
                                    const int* __restrict__ R, int nR, const double* __restrict__ eps, int NG,
                                    int ig0, c2<T>* __restrict__ N) {
  const int64_t total = (int64_t)nL * nR;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    double2 d = make_double2(0.0, 0.0);
    for (int z = 0; z < nsplit; ++z) {
      const double2 v = Dp[(int64_t)z * total + id];
      d.x += v.x;
      d.y += v.y;
    }
    const int a = (int)(id / nR), b = (int)(id % nR);
    const double de = eps[R[b]] - eps[L[a]];
    N[id * NG + ig0] = mk<T>((T)(d.y / de), (T)(-d.x / de));  // -i D / de
  }
}

static int dipole_rows(int nL) { return nL <= 16 ? 16 : nL <= 32 ? 32 : 64; }

static int dipole_nsplit(int nL, int nR, int K) {
  const int TL = dipole_rows(nL);
  const int tiles = ((nR + OT - 1) / OT) * ((nL + TL - 1) / TL);
  return std::max(1, std::min((K + 255) / 256, (2 * 152 + tiles - 1) / tiles));
}

int64_t optical_scratch_elems(int nL, int nR, int npw, int KP) {
  return (int64_t)nR * KP + (int64_t)dipole_nsplit(nL, nR, npw + KP) * nL * nR;
}

template <typename T>
cudaError_t launch_optical_head(const double2* C, int npw, const double* s, const double2* P, int KP,
                                const double2* Qn, double2* scratch, const int* L, int nL, const int* R, int nR,
                                const double* eps, int NG, int ig0, c2<T>* N, cudaStream_t st) {
  if (nL == 0 || nR == 0) return cudaSuccess;
  // scratch: Y [nR][KP], then the K-split partials [nsplit][nL][nR]
  const int kp = P ? KP : 0;
  double2* Y = scratch;
  double2* Dp = scratch + (int64_t)nR * kp;
  if (P) {
    const int64_t total = (int64_t)nR * KP;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    optical_paw_y_kernel<<<blocks, 256, 0, st>>>(P, KP, Qn, R, nR, Y);
  }
  const int K = npw + kp;
  const int TL = dipole_rows(nL);
  const int nsplit = dipole_nsplit(nL, nR, K);
  const int kslice = ((K + nsplit - 1) / nsplit + OK - 1) / OK * OK;
  dim3 grid((nR + OT - 1) / OT, (nL + TL - 1) / TL, nsplit);
  if (TL == 16)
    optical_dipole_kernel<T, 1><<<grid, 256, 0, st>>>(C, npw, s, P, KP, Y, L, nL, R, nR, kslice, Dp);
  else if (TL == 32)
    optical_dipole_kernel<T, 2><<<grid, 256, 0, st>>>(C, npw, s, P, KP, Y, L, nL, R, nR, kslice, Dp);
  else
    optical_dipole_kernel<T, 4><<<grid, 256, 0, st>>>(C, npw, s, P, KP, Y, L, nL, R, nR, kslice, Dp);
  const int64_t total = (int64_t)nL * nR;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  optical_head_kernel<T><<<blocks, 256, 0, st>>>(Dp, nsplit, L, nL, R, nR, eps, NG, ig0, N);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- adjoint of the head
// The head n0_nm = -i D_nm / (e_m - e_n) replaced the G = 0 pair densities, so
// dE/dn0 (the G = 0 column of Nbar) flows back through the dipole matrix D of
// Eq. 13 instead of the transforms and the PAW term.  With
//   b_nm = i Nbar_nm(0) / (e_m - e_n),   dE = Re sum conj(b) dD,
// the PyTorch-convention gradients (g = 2 dE/dconj(z)) are
//   g_C_m(Q) += sum_n -i b_nm s(Q) C_n(Q),    g_C_n(Q) += sum_m i conj(b_nm) s(Q) C_m(Q),
//   g_P_mj += sum_n b_nm sum_i P_ni conj(Qn_ij),  g_P_ni += sum_m conj(b_nm) sum_j Qn_ij P_mj,
// all FP64.

// b[a][r] = i Nbar[(a nR + r) NG + ig0] / (e_R[r] - e_L[a]); that Nbar column is cleared
template <typename T>
__global__ void optical_adj_b_kernel(c2<T>* __restrict__ Nbar, int NG, int ig0, const int* __restrict__ L, int nL,
                                     const int* __restrict__ R, int nR, const double* __restrict__ eps,
                                     double2* __restrict__ bm) {
  const int64_t total = (int64_t)nL * nR;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(id / nR), r = (int)(id % nR);
    const c2<T> nb = Nbar[id * NG + ig0];
    const double de = eps[R[r]] - eps[L[a]];
    bm[id] = make_double2(-(double)nb.y / de, (double)nb.x / de);  // i nb / de
    Nbar[id * NG + ig0] = mk<T>(0, 0);
  }
}

// out[ro(i) ldo + j] += sum_k coef(i, k) op_x(X[rx(k) sxk + j sxj]) sc(j), i < M, j < N, k < K,
// coef(i, k) = mult op_a(A[ra(i) sai + k sak]); ro, ra, rx are optional row
// lists, op_* an optional conjugation, sc an optional real column scale.
struct AdjGemm {
  double2* out;
  const int* ro;
  int64_t ldo;
  const double2* A;
  const int* ra;
  int64_t sai, sak;
  double2 mult;
  int conj_a;
  const double2* X;
  const int* rx;
  int64_t sxk, sxj;
  int conj_x;
  const double* sc;
  int M, N, K;
};

__global__ void __launch_bounds__(256) optical_adj_gemm_kernel(const AdjGemm g) {
  __shared__ double2 As[16][17];
  __shared__ double2 Xs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
  double2 acc = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < g.K; k0 += 16) {
    {
      // coefficient tile: row i0 + ty, column k0 + tx
      const int k = k0 + tx;
      double2 v = make_double2(0.0, 0.0);
      if (i < g.M && k < g.K) {
        const int64_t r = g.ra ? g.ra[i] : i;
        v = g.A[r * g.sai + (int64_t)k * g.sak];
        if (g.conj_a) v.y = -v.y;
        v = make_double2(g.mult.x * v.x - g.mult.y * v.y, g.mult.x * v.y + g.mult.y * v.x);
      }
      As[ty][tx] = v;
    }
    {
      // X tile: row k0 + ty, column j0 + tx
      const int k = k0 + ty;
      double2 v = make_double2(0.0, 0.0);
      if (k < g.K && j < g.N) {
        const int64_t r = g.rx ? g.rx[k] : k;
        v = g.X[r * g.sxk + (int64_t)j * g.sxj];
        if (g.conj_x) v.y = -v.y;
      }
      Xs[ty][tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) cmac<double>(acc, As[ty][kk], Xs[kk][tx]);
    __syncthreads();
  }
  if (i < g.M && j < g.N) {
    const double f = g.sc ? g.sc[j] : 1.0;
    double2* o = g.out + (g.ro ? (int64_t)g.ro[i] : (int64_t)i) * g.ldo + j;
    double2 v = *o;
    v.x += f * acc.x;
    v.y += f * acc.y;
    *o = v;
  }
}

static cudaError_t adj_gemm(const AdjGemm& g, cudaStream_t st) {
  if (g.M == 0 || g.N == 0 || g.K == 0) return cudaSuccess;
  dim3 grid((g.N + 15) / 16, (g.M + 15) / 16);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  optical_adj_gemm_kernel<<<grid, 256, 0, st>>>(g);
  return cudaGetLastError();
}

int64_t optical_adj_scratch_elems(int nL, int nR, int KP) { return (int64_t)nL * nR + (int64_t)(nL + nR) * KP; }

template <typename T>
cudaError_t launch_optical_adjoint(c2<T>* Nbar, int NG, int ig0, const int* L, int nL, const int* R, int nR,
                                   const double* eps, const double2* C, int npw, const double* s, const double2* P,
                                   int KP, const double2* Qn, double2* scratch, double2* gC, double2* gP,
                                   cudaStream_t st) {
  if (nL == 0 || nR == 0) return cudaSuccess;
  double2* bm = scratch;                       // [nL][nR]
  double2* Y = bm + (int64_t)nL * nR;          // [nL][KP]
  double2* Z = Y + (int64_t)nL * KP;           // [nR][KP]
  {
    const int64_t total = (int64_t)nL * nR;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    optical_adj_b_kernel<T><<<blocks, 256, 0, st>>>(Nbar, NG, ig0, L, nL, R, nR, eps, bm);
  }
  const double2 one = make_double2(1.0, 0.0), mi = make_double2(0.0, -1.0), pi = make_double2(0.0, 1.0);
  cudaError_t e;
  // g_C_m(Q) += sum_n -i b_nm s(Q) C_n(Q): rows R, coef(r, a) = -i b[a][r]
  if ((e = adj_gemm({gC, R, npw, bm, nullptr, 1, nR, mi, 0, C, L, npw, 1, 0, s, nR, npw, nL}, st)) != cudaSuccess)
    return e;
  // g_C_n(Q) += sum_m i conj(b_nm) s(Q) C_m(Q): rows L, coef(a, r) = i conj(b[a][r])
  if ((e = adj_gemm({gC, L, npw, bm, nullptr, nR, 1, pi, 1, C, R, npw, 1, 0, s, nL, npw, nR}, st)) != cudaSuccess)
    return e;
  if (P && Qn && gP && KP > 0) {
    if ((e = cudaMemsetAsync(Y, 0, sizeof(double2) * (size_t)(nL + nR) * KP, st)) != cudaSuccess) return e;
    // Y[a][j] = sum_i P[L[a]][i] conj(Qn[i][j])
    if ((e = adj_gemm({Y, nullptr, KP, P, L, KP, 1, one, 0, Qn, nullptr, KP, 1, 1, nullptr, nL, KP, KP}, st)) !=
        cudaSuccess)
      return e;
    // g_P[R[r]][j] += sum_a b[a][r] Y[a][j]
    if ((e = adj_gemm({gP, R, KP, bm, nullptr, 1, nR, one, 0, Y, nullptr, KP, 1, 0, nullptr, nR, KP, nL}, st)) !=
        cudaSuccess)
      return e;
    // Z[r][i] = sum_j P[R[r]][j] Qn[i][j]
    if ((e = adj_gemm({Z, nullptr, KP, P, R, KP, 1, one, 0, Qn, nullptr, 1, KP, 0, nullptr, nR, KP, KP}, st)) !=
        cudaSuccess)
      return e;
    // g_P[L[a]][i] += sum_r conj(b[a][r]) Z[r][i]
    if ((e = adj_gemm({gP, L, KP, bm, nullptr, nR, 1, one, 1, Z, nullptr, KP, 1, 0, nullptr, nL, KP, nR}, st)) !=
        cudaSuccess)
      return e;
  }
  return cudaGetLastError();
}

template cudaError_t launch_optical_adjoint<float>(float2*, int, int, const int*, int, const int*, int, const double*,
                                                   const double2*, int, const double*, const double2*, int,
                                                   const double2*, double2*, double2*, double2*, cudaStream_t);
template cudaError_t launch_optical_adjoint<double>(double2*, int, int, const int*, int, const int*, int,
                                                    const double*, const double2*, int, const double*, const double2*,
                                                    int, const double2*, double2*, double2*, double2*, cudaStream_t);

// dst[i] += src[i]
__global__ void add_c128_kernel(double2* __restrict__ dst, const double2* __restrict__ src, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    dst[i].x += src[i].x;
    dst[i].y += src[i].y;
  }
}

cudaError_t launch_add_c128(double2* dst, const double2* src, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  add_c128_kernel<<<blocks, 256, 0, st>>>(dst, src, n);
  return cudaGetLastError();
}

template cudaError_t launch_optical_head<float>(const double2*, int, const double*, const double2*, int,
                                                const double2*, double2*, const int*, int, const int*, int,
                                                const double*, int, int, float2*, cudaStream_t);
template cudaError_t launch_optical_head<double>(const double2*, int, const double*, const double2*, int,
                                                 const double2*, double2*, const int*, int, const int*, int,
                                                 const double*, int, int, double2*, cudaStream_t);

}  // namespace rpa

// ---------------------------------------------------------------- IBZ -> BZ symmetry (Eq. 9, steps 4 and 7)
namespace rpa {

__global__ void conj_kernel(double2* __restrict__ x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i].y = -x[i].y;
}

// out[n][off[a] + i] = sum_j D[doff[a] + i ni + j] P[n][off[src[a]] + j], conjugated if tr
__global__ void rotate_P_kernel(const double2* __restrict__ P, int nb, int KP, int natoms, const int* __restrict__ meta,
                                const double2* __restrict__ D, int tr, double2* __restrict__ out) {
  // meta: off[natoms], src[natoms], ni[natoms], doff[natoms], atom_of[KP], idx_in[KP]
  const int* off = meta;
  const int* src = off + natoms;
  const int* nis = src + natoms;
  const int* doff = nis + natoms;
  const int* atom_of = doff + natoms;
  const int* idx_in = atom_of + KP;
  const int64_t total = (int64_t)nb * KP;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(id % KP);
    const int64_t n = id / KP;
    const int a = atom_of[k], i = idx_in[k], ni = nis[a];
    const double2* ps = P + n * KP + off[src[a]];
    const double2* d = D + doff[a] + (int64_t)i * ni;
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < ni; ++j) cmac<double>(acc, d[j], ps[j]);
    if (tr) acc.y = -acc.y;
    out[id] = acc;
  }
}

// C[n][q] *= ph[q] for nb bands of npw plane waves
__global__ void phase_kernel(double2* __restrict__ C, int64_t nb, int npw, const double2* __restrict__ ph) {
  const int64_t total = nb * npw;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = C[i], b = ph[i % npw];
    C[i] = make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
  }
}

cudaError_t launch_phase(double2* C, int64_t nb, int npw, const double2* ph, cudaStream_t s) {
  const int64_t n = nb * npw;
  if (n == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  phase_kernel<<<blocks, 256, 0, s>>>(C, nb, npw, ph);
  return cudaGetLastError();
}

cudaError_t launch_conj(double2* x, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  conj_kernel<<<blocks, 256, 0, s>>>(x, n);
  return cudaGetLastError();
}

cudaError_t launch_rotate_P(const double2* P, int nb, int KP, int natoms, const int* meta, const double2* D, int tr,
                            double2* out, cudaStream_t s) {
  const int64_t total = (int64_t)nb * KP;
  if (total == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  rotate_P_kernel<<<blocks, 256, 0, s>>>(P, nb, KP, natoms, meta, D, tr, out);
  return cudaGetLastError();
}

}  // namespace rpa
