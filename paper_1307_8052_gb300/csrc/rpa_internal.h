// Internal declarations shared by the host runtime and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

namespace rpa {

template <typename T> struct vec2;
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<double> { using type = double2; };
template <typename T> using c2 = typename vec2<T>::type;

template <typename T> __host__ __device__ inline c2<T> mk(T re, T im) { c2<T> r; r.x = re; r.y = im; return r; }

// acc += a * b
template <typename T> __device__ __forceinline__ void cmac(c2<T>& acc, c2<T> a, c2<T> b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc += a * conj(b)
template <typename T> __device__ __forceinline__ void cmac_cj(c2<T>& acc, c2<T> a, c2<T> b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.y, b.x, acc.y); acc.y = fma(-a.x, b.y, acc.y);
}
// conj(a) * b
template <typename T> __device__ __forceinline__ c2<T> cj_mul(c2<T> a, c2<T> b) {
  return mk<T>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// ---------------------------------------------------------------- kernels
// Generic pruned DFT along one axis of a [batch][A][Lin][B] array:
//   out[b][a][o][c] = sum_i in[b][a][i][c] * exp(sign * 2 pi i (in_off+i)(out_off+o) / N)
template <typename T>
cudaError_t launch_dft_axis(const c2<T>* in, c2<T>* out, int64_t batch, int A, int Lin, int Lout,
                            int B, int N, int in_off, int out_off, int sign, cudaStream_t s);

// Scatter plane-wave coefficients (double complex [nb][npw]) into a zeroed
// Miller box [nb][box] at the flat positions pos[npw].
template <typename T>
cudaError_t launch_scatter_box(const double2* C, int nb, int npw, const int* pos, int64_t box,
                               c2<T>* out, cudaStream_t s);

// Pair densities, stage A: fused conj(u_n) u_m product and pruned DFT along
// the slowest grid axis.  Chunk slot pl is pair (pl % nrow) * nR + p0 + pl / nrow
// of the rectangle L x R (a-major): nrow rows of np / nrow columns from p0,
// rows fastest; nrow = 1 is the contiguous range p0 .. p0+np-1.
template <typename T>
cudaError_t launch_pd_stageA(const c2<T>* Uk, const c2<T>* Ukp, int64_t Nr, int N1, int N23,
                             const int* Lidx, const int* Ridx, int nR, int64_t p0, int np, int nrow,
                             const c2<T>* tw, int n1, c2<T>* T1, cudaStream_t s);

// Twiddle matrices tw[oc][j][o] = exp(-2 pi i (lo + 16 oc + o) j / N) for the
// n pruned outputs of an N-point axis (16 outputs per chunk), FP64-accurate.
template <typename T>
cudaError_t launch_twiddle_matrix(c2<T>* tw, int N, int lo, int n, cudaStream_t s);

// Pair densities, stage B: pruned DFT along the middle axis,
//   T2[pl][o1][o2][j3] = sum_j2 T1[pl][o1][j2][j3] exp(-2 pi i (g2lo+o2) j2 / N2).
// Stages A and B with the N-point axis factorised as (N / L) x L (two-level
// pruned DFT; factored_radix picks L, 0 = keep the direct form); the table
// comes from launch_twiddle_factored (L^2 + (N / L) * 16 entries).
int factored_radix(int N, int n);
template <typename T>
cudaError_t launch_twiddle_factored(c2<T>* tw, int N, int L, int lo, int n, cudaStream_t s);
template <typename T>
cudaError_t launch_pd_stageA_fact(const c2<T>* Uk, const c2<T>* Ukp, int64_t Nr, int N1, int N23, const int* Lidx,
                                  const int* Ridx, int nR, int64_t p0, int np, int nrow, const c2<T>* twf, int L,
                                  int n1, c2<T>* T1, cudaStream_t s);
template <typename T>
cudaError_t launch_pd_stageB_fact(const c2<T>* T1, c2<T>* T2, int np, int n1, int N2, int N3, const c2<T>* twf, int L,
                                  int n2, cudaStream_t s);

template <typename T>
cudaError_t launch_pd_stageB(const c2<T>* T1, c2<T>* T2, int np, int n1, int N2, int N3, const c2<T>* tw, int n2,
                             cudaStream_t s);

// Pair densities, stage C: DFT along the fastest axis evaluated on the sphere
// points g = G + G0, 1/Nr normalisation, write N[p][NG].
template <typename T>
cudaError_t launch_pd_stageC(const c2<T>* T2, int np, int n1, int n2, int N3, const int* gfft,
                             int NG, int g1lo, int g2lo, double inv_nr, int64_t p0, int nrow, int nR,
                             const c2<T>* tw3, c2<T>* Nout, cudaStream_t s);
// tw[t] = exp(2 pi i t / N), t < N (FP64-accurate), for stage C's tw3 (or null:
// every block forms its own).
template <typename T>
cudaError_t launch_twiddle_line(c2<T>* tw, int N, cudaStream_t s);

// Pair densities, stages B and C fused per (pair, slab of OB first-axis
// outputs): the middle-axis DFT into shared memory, then the fastest axis on
// the sphere points of the slab (g1start[o] = first sphere point with
// g1 - g1lo >= o); bit-identical to stage B followed by stage C.
// pd_stageBC_slab gives the slab height that fits (0: use stages B and C).
template <typename T>
cudaError_t launch_pd_stageBC(const c2<T>* T1, int np, int n1, int N2, int N3, const c2<T>* tw, int n2,
                              const int* gfft, const int* g1start, int OB, int NG, int g1lo, int g2lo, double inv_nr,
                              int64_t p0, c2<T>* Nout, cudaStream_t s);
template <typename T>
int pd_stageBC_slab(int n1, int n2, int N2, int N3);
cudaError_t launch_g1start(const int* gfft, int NG, int g1lo, int n1, int* out, cudaStream_t s);

// PAW term of a block: N[(a nR + b)][g] += sum_kp Pm[b][kp] R[a][kp][g].
template <typename T>
cudaError_t launch_paw_gemm(const c2<T>* R, const c2<T>* Pm, int KP, int nL, int nR, int NG, c2<T>* N,
                            cudaStream_t s);

// PAW factor R_a[aL][kp][G] = sum_i conj(P_n,(a,i)) Q^a_ij(G), FP64 arithmetic.
template <typename T>
cudaError_t launch_paw_R(const double2* Pk, int KP, const int* Lidx, int nL, const double2* Q,
                         const int* atom_of_kp, const int* idx_in_atom, const int* atom_off,
                         const int64_t* q_off, const int* nproj, int NG, c2<T>* R, cudaStream_t s);

// Gather projections P[m][kp] of the R set into working precision.
template <typename T>
cudaError_t launch_gather_P(const double2* P, int KP, const int* Ridx, int nR, c2<T>* out,
                            cudaStream_t s);

// Pair parameters: d_p = e_n - e_m and df_p = max(f_n - f_m, 0).
cudaError_t launch_pair_params(const double* ek, const double* fk, const double* ekp,
                               const double* fkp, const int* Lidx, int nL, const int* Ridx, int nR,
                               double* d, double* df, cudaStream_t s);

// Real pair weights of Eq. 3 (time-reversal combined), per frequency:
//   wgt[j][p] = pref * df_p * 2 d_p / (w_j^2 + d_p^2), computed in FP64.
cudaError_t launch_pair_weights(const double* d, const double* df, const double* omega, int nw, int64_t P,
                                double pref, double* w64, float* w32, cudaStream_t s);

// Hermitian rank-k update on CUDA cores (FP64 or FP32 with compensated folds):
//   chi[w][i][j] += sum_p wgt[w][p] N[p][i] conj(N[p][j]) for lower-triangle tiles.
template <typename T>
cudaError_t launch_herk_simt_w(const c2<T>* N, int64_t P, int NG, const T* wgt, int nw, double2* chi,
                               cudaStream_t s);

// Upper triangle from lower: chi[w][i][j] = conj(chi[w][j][i]) for i < j.
cudaError_t launch_hermitian_fill(double2* chi, int nw, int NG, cudaStream_t s);

// Optical limit (k_optical.cu): G = 0 column of a block of pair densities at
// q = 0 from q^.<psi_n|grad|psi_m> (plane-wave part with s[Q] = q^.(k+Q),
// PAW part from the dense q^.Q_grad matrix Qn [KP][KP]); scratch holds
// optical_scratch_elems(nL, nR, npw, KP) complex FP64 elements.
int64_t optical_scratch_elems(int nL, int nR, int npw, int KP);
template <typename T>
cudaError_t launch_optical_head(const double2* C, int npw, const double* s, const double2* P, int KP,
                                const double2* Qn, double2* scratch, const int* L, int nL, const int* R, int nR,
                                const double* eps, int NG, int ig0, c2<T>* N, cudaStream_t st);

// Adjoint of the optical head (k_optical.cu): the G = 0 column of Nbar flows
// back through the dipole matrix into the FP64 gradients of C (gC [nb][npw])
// and P (gP [nb][KP]) of the q = 0 point's orbital set, and is then cleared;
// scratch holds optical_adj_scratch_elems(nL, nR, KP) complex FP64 elements.
int64_t optical_adj_scratch_elems(int nL, int nR, int KP);
template <typename T>
cudaError_t launch_optical_adjoint(c2<T>* Nbar, int NG, int ig0, const int* L, int nL, const int* R, int nR,
                                   const double* eps, const double2* C, int npw, const double* s, const double2* P,
                                   int KP, const double2* Qn, double2* scratch, double2* gC, double2* gP,
                                   cudaStream_t st);
// dst[i] += src[i] (complex FP64)
cudaError_t launch_add_c128(double2* dst, const double2* src, int64_t n, cudaStream_t st);

// IBZ -> BZ symmetry (k_optical.cu): conjugation of coefficients, and rotation
// of projections out[n][a][i] = sum_j D^a_ij P[n][src(a)][j] (conjugated if tr);
// meta = off[natoms], src[natoms], ni[natoms], doff[natoms], atom_of[KP], idx_in[KP].
cudaError_t launch_conj(double2* x, int64_t n, cudaStream_t s);
cudaError_t launch_phase(double2* C, int64_t nb, int npw, const double2* ph, cudaStream_t s);
cudaError_t launch_rotate_P(const double2* P, int nb, int KP, int natoms, const int* meta, const double2* D, int tr,
                            double2* out, cudaStream_t s);

// Complex elements of the work buffer run_logdet needs: the factor and the
// inverses of its diagonal blocks.
int64_t logdet_work_elems(int nw, int NG);

// One matrix of a batched float-float log-det (one frequency of one
// instance): slices of that instance's run_logdet work buffer (the matrix, the
// two CB x CB inverses, the first [NG][CB] panel) and its outputs.
struct LdMat {
  double2* A;
  double2* Linv;
  float4* Linv_ff;
  float4* Lp;
  const double2* chi;  // chi0 of this frequency [NG][NG]
  const double* v;     // Coulomb kernel [NG]
  double* logdet;      // ln det of this frequency
  double* trace;       // tr(v chi0) of this frequency
  int* flag;           // the instance's non-HPD flag
  int NG;
};
// Float-float log-dets of nmat matrices (descriptors in device memory) in one
// sequence of launches on s (no look-ahead); maxNG = the largest NG.
cudaError_t run_logdet_batch(const LdMat* d, int nmat, int maxNG, cudaStream_t s, int64_t* launches);
// LdMat of frequency w with the work-buffer slices filled in (outputs unset).
LdMat logdet_mat(double2* work, int nw, int NG, int w);

// Second stream and events of the look-ahead factorisation (float-float mode).
struct LogdetStreams {
  cudaStream_t s2;
  cudaEvent_t ev_t, ev_u;
};

// Log-det of 1 - v^1/2 chi v^1/2 by blocked Cholesky in FP64, batched over w:
// per-w ln det in logdet, tr(v^1/2 chi v^1/2) in trace, pivot failure in flag.
// ff_update evaluates the trailing updates in float-float arithmetic; with la
// it also factorises the next panel beside the rest of the current update.
// formed (optional) is recorded on s once chi has been read (matrix formed,
// trace taken), after which the caller may reuse the chi buffer.
cudaError_t run_logdet(const double2* chi, const double* v, int nw, int NG, double2* work,
                       double* logdet, double* trace, int* flag, bool ff_update, cudaStream_t s,
                       int64_t* launches, const LogdetStreams* la = nullptr, cudaEvent_t formed = nullptr);

}  // namespace rpa
