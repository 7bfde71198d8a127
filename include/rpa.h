/*
 * rpa.h -- C ABI of the GB300 library for the non-interacting response
 * function chi0_GG'(q, i w) and the RPA correlation energy E_c.
 *
 * The operations follow Yan, Li and O'Grady, "Graphics processing unit
 * acceleration of the random phase approximation in the projector augmented
 * wave method":
 *   - chi0 by the sum over states, Eq. 3, accumulated as the grouped
 *     ("multi-u") Hermitian rank-k update of Eq. 17 for every frequency;
 *   - pair densities n_nm(G) of Eq. 4 from real-space orbital products and a
 *     forward Fourier transform (Eq. 10), gathered on the response G sphere
 *     (Table 1 steps 5-6), plus the PAW augmentation of Eq. 6 (steps 7-9);
 *   - E_c of Eqs. 1-2: sum over q of w_q, over Gauss-Legendre frequencies of
 *     W_j / (2 pi) [ln det(1 - v^1/2 chi0 v^1/2) + tr(v^1/2 chi0 v^1/2)]
 *     (Table 1 step 13);
 *   - the optical limit q -> 0 of Eqs. 12-14 (rpa_set_optical), the IBZ -> BZ
 *     symmetry of Eq. 9 (rpa_set_orbitals_sym), the gradient of E_c
 *     (rpa_energy_backward) and the inverse dielectric matrix
 *     (rpa_epsilon_inv); many independent q-points or cells can be batched
 *     into one CUDA graph (rpa_graph_*).
 *
 * Conventions (all functions):
 *   - Complex arrays are interleaved (re, im) doubles.
 *   - Lattice vectors are the rows of cell[9] (bohr); k, q are given in
 *     reduced coordinates of the reciprocal lattice; Miller indices are int32
 *     triples.  A grid point j = (j1, j2, j3) of the N1 x N2 x N3 grid sits at
 *     r = sum_i (j_i / N_i) a_i.
 *   - Orbital coefficients follow Eq. 8: psi_nk(r) = Omega^-1/2 sum_Q C_nk(Q)
 *     exp(i (k+Q).r) with sum_Q |C_nk(Q)|^2 = 1.
 *   - Bulk arrays documented "host or device" (C, P, Q, D, chi0 and
 *     gradient outputs) may be host, managed or CUDA device memory; the
 *     library copies what it keeps and never retains a caller pointer after a
 *     call returns.  Device outputs are written in order on the context's
 *     stream, host outputs are complete when the call returns.  Every other
 *     pointer (index lists, frequencies, weights, small parameter arrays,
 *     scalar outputs) is read or written by the host: pageable, pinned or
 *     managed memory; CUDA device memory there is RPA_ERR_ARG.
 *     rpa_logdet_noalloc, which takes device memory, states its own rule.
 *   - Every call returns an rpa_status; rpa_last_error() gives a message.
 *     No call aborts the process or traps on the device.  A context is not
 *     thread-safe: use one context per host thread.
 */
#ifndef RPA_GB300_H
#define RPA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rpa_ctx rpa_ctx;

typedef enum {
  RPA_OK = 0,
  RPA_ERR_ARG = 1,      /* invalid argument (sizes, indices, aliasing grid) */
  RPA_ERR_OOM = 2,      /* device allocation failed */
  RPA_ERR_CUDA = 3,     /* CUDA runtime/driver error */
  RPA_ERR_NOT_HPD = 4,  /* 1 - v^1/2 chi0 v^1/2 not Hermitian positive definite */
  RPA_ERR_TIMEOUT = 5,  /* a bounded device-side wait gave up */
  RPA_ERR_STATE = 6     /* call out of order (e.g. missing orbitals) */
} rpa_status;

/* Arithmetic of the rank-k update (Eq. 17) and of the pair densities.
 * RPA_FP64   : everything in FP64.
 * RPA_FP32   : pair densities and rank-k update in FP32 (CUDA cores), with
 *              compensated FP32 folding of partial sums; chi0 held in FP64.
 * RPA_BF16X2 : pair densities in FP32; rank-k update on the tensor cores with
 *              each operand split into two bfloat16 terms (hi + lo, three
 *              products), FP32 accumulation in tensor memory, FP64 chi0.
 * RPA_BF16X3 : as BF16X2 with three bfloat16 terms (hi + mid + lo, about
 *              24 bits per operand) and six products (hh, hm, mh, mm, hl, lh).
 * In every mode the PAW factor R_n(j, G) = sum_i conj(P_ni) Q_ij(G) is formed
 * in FP64 and stored in the mode's working precision; the PAW product
 * sum_j P_mj R_n(j, G) runs in FP32 on the CUDA cores in the mixed modes (or
 * on the tensor cores, RPA_TUNE_PAW_TC).  The log-det is FP64 in RPA_FP64 and
 * float-float (about 44 bits, FP64 pivots) in the other modes
 * (RPA_TUNE_LOGDET); the frequency quadrature is FP64. */
typedef enum {
  RPA_FP64 = 0,
  RPA_FP32 = 1,
  RPA_BF16X2 = 2,
  RPA_BF16X3 = 3
} rpa_precision;

typedef struct {
  double cell[9];      /* lattice vectors a1, a2, a3 as rows, bohr */
  int32_t grid[3];     /* real-space grid N1, N2, N3 of Eq. 10 */
  double ecut_chi;     /* response cutoff: G with |q+G|^2 / 2 <= ecut_chi (Ha) */
  double spin_factor;  /* s in s / (Omega N_k); 2 for spin-paired orbitals */
  int32_t nk_bz;       /* N_k of the Brillouin-zone average */
  int32_t precision;   /* rpa_precision */
  int32_t device;      /* CUDA device ordinal */
  void* stream;        /* cudaStream_t to order work on; NULL: library stream */
} rpa_params;

/* Creates a context on params->device holding the fixed inputs of the
 * calculation (Table 1: the cell and real-space grid of Eqs. 8 and 10, the
 * response cutoff of Sec. 2.1, the prefactor s / (Omega N_k) of Eq. 3).
 * Validates the cell (non-singular),
 * grid (each N_i in [2, 768]), ecut_chi > 0, spin_factor > 0, nk_bz >= 1 and
 * the precision.  *out receives the context; RPA_ERR_ARG on bad parameters,
 * RPA_ERR_CUDA if the device cannot be used. */
rpa_status rpa_create(const rpa_params* params, rpa_ctx** out);

/* Releases every device allocation of the context (no counterpart in the
 * paper).  NULL is ignored. */
void rpa_destroy(rpa_ctx* ctx);

/* Message of the last failing call on this context (never NULL; no
 * counterpart in the paper). */
const char* rpa_last_error(const rpa_ctx* ctx);

/* Gauss-Legendre frequency grid (Sec. 2.1, 16 points in the paper) mapped to
 * [0, inf) by w = w0 (1 + x) / (1 - x): omega[n] nodes, W[n] weights with
 * int_0^inf f(w) dw ~ sum_j W_j f(omega_j).  Host pointers.  n in [1, 1024]. */
rpa_status rpa_gauss_legendre(int32_t n, double omega0, double* omega, double* W);

/* Orbital set kidx (Eq. 8; Table 1 step 2): the k-point k_red[3], nbands
 * bands on npw plane waves with Miller indices miller[npw][3], coefficients
 * C[nbands][npw] (complex), eigenvalues eps[nbands] (Ha) and occupations
 * f[nbands] in [0, 1] per spin channel.  Replaces a previous set kidx (and
 * drops its projections).  kidx in [0, 4096).  Miller indices must be
 * distinct.  C may be host or device memory; miller, eps, f are host. */
rpa_status rpa_set_orbitals(rpa_ctx* ctx, int32_t kidx, const double k_red[3],
                            int32_t nbands, int32_t npw, const int32_t* miller,
                            const double* C, const double* eps, const double* f);

/* IBZ -> BZ symmetry (Eq. 9; Table 1 steps 4 and 7): orbital set kidx becomes
 * the set src transformed by a crystal symmetry {T|tau},
 * psi'(r) = psi(T^-1 (r - tau)), with optional time reversal psi -> conj(psi).
 * M[9] (row-major, integers) is T on reduced reciprocal coordinates: k' = M k,
 * and every plane wave Q -> M Q keeps its coefficient times
 * exp(-2 pi i (M (k+Q)).tau), tau[3] the fractional translation in reduced
 * real-space coordinates (NULL = 0).  time_reversal != 0 then negates k' and
 * Q' and conjugates the coefficients.  M must be unimodular and keep the
 * reciprocal metric (M^T B B^T M = B B^T), else RPA_ERR_ARG.  Eigenvalues and
 * occupations are copied.  If src has projections, natoms must equal its
 * atom count and P'[n][a][i] = sum_j D^a_ij P[n][atom_map[a]][j] (conjugated
 * under time reversal), D atom after atom [ni][ni] complex, host or device
 * (lattice-vector phases of the projectors belong in D).  kidx != src; the
 * source is not modified. */
rpa_status rpa_set_orbitals_sym(rpa_ctx* ctx, int32_t kidx, int32_t src, const int32_t* M, const double* tau,
                                int32_t time_reversal, int32_t natoms, const int32_t* atom_map, const double* D);

/* PAW projections of set kidx (Eq. 6; Table 1 step 7):
 * P[nbands][sum_a nproj[a]] (complex) with P_ni = <p~^a_i | psi~_nk>, atoms
 * in order.  nproj[a] in [1, 64].  P host or device. */
rpa_status rpa_set_paw(rpa_ctx* ctx, int32_t kidx, int32_t natoms,
                       const int32_t* nproj, const double* P);

/* q-point iq (Eq. 2; Table 1 step 14): q_red[3] and its nk transitions
 * k -> k+q, each given as (k_of[t], kq_of[t], G0[t][3]) meaning the orbitals
 * at k are set k_of[t] and k + q = k' + G0 with k' the k-point of set
 * kq_of[t].  Builds the response sphere {G : |q+G|^2/2 <= ecut_chi} in
 * Miller-lexicographic order (first index slowest) and the Coulomb kernel
 * v_G = 4 pi / |q+G|^2 (0 where q + G = 0).  *ng_out (nullable) receives NG.
 * The referenced orbital sets must exist; the grid must be large enough that
 * the Fourier route of Eq. 10 has no aliasing for them (RPA_ERR_ARG
 * otherwise).  iq in [0, 4096).  All pointers host. */
rpa_status rpa_set_qpoint(rpa_ctx* ctx, int32_t iq, const double q_red[3],
                          int32_t nk, const int32_t* k_of, const int32_t* kq_of,
                          const int32_t* G0, int32_t* ng_out);

/* The response sphere of q-point iq: the reciprocal lattice vectors G that
 * index chi0_GG'(q) and v_G(q), |q+G|^2/2 <= E_cut (Sec. 2.1; Table 1 step 6
 * gathers the pair densities onto them).  *ng receives NG and, if
 * miller_out != NULL, miller_out[ng][3] their Miller indices in the order
 * chi0, epsilon^-1 and the Q^a_ij input use (Miller-lexicographic, first
 * index slowest).  Host pointers.  RPA_ERR_STATE if q-point iq is not set. */
rpa_status rpa_gvectors(const rpa_ctx* ctx, int32_t iq, int32_t* ng,
                        int32_t* miller_out);

/* The same sphere without a context or a GPU (host arithmetic only): for the
 * lattice rows cell[9] (bohr), q_red[3] (reduced) and ecut_chi (Ha), *ng
 * receives NG, miller_out[ng][3] (nullable) the Miller indices in the order
 * rpa_set_qpoint builds for the same cell, q and cutoff, and v_out[ng]
 * (nullable) the Coulomb kernel v_G = 4 pi / |q+G|^2 of Sec. 2.2, 0 where
 * q + G = 0.  Call with cap = 0 and NULL outputs to size them; a non-NULL
 * output with cap < NG is RPA_ERR_ARG (*ng is still set).  NG = 0 is a valid
 * answer.  RPA_ERR_ARG for NULL cell/q_red/ng, a singular cell, non-finite q,
 * ecut_chi <= 0 or a Miller search box over 2^28 points. */
rpa_status rpa_response_sphere(const double cell[9], const double q_red[3],
                               double ecut_chi, int32_t cap, int32_t* ng,
                               int32_t* miller_out, double* v_out);

/* PAW augmentation functions of q-point iq (Eq. 6, Q^a_ij(q+G)):
 * atom after atom a block Q[ni][ni][NG] (complex), G in rpa_gvectors order.
 * natoms/nproj must match the projections of every orbital set used by iq.
 * Q host or device. */
rpa_status rpa_set_paw_Q(rpa_ctx* ctx, int32_t iq, int32_t natoms,
                         const int32_t* nproj, const double* Q);

/* Optical limit q -> 0 at q-point iq (Eqs. 12-14).  iq must have q = 0 and
 * only k -> k transitions without umklapp.  The G = 0 pair density of every
 * pair becomes its q -> 0 limit per unit |q| along the direction qdir[3]
 * (Cartesian, normalised by the library),
 *   n_nm(0) = -i q^.<psi_n|grad|psi_m> / (e_m - e_n),
 *   <psi_n|grad|psi_m> = i sum_Q conj(C_n(Q)) (k+Q) C_m(Q)
 *                        + sum_a sum_ij conj(P_ni) P_mj Qgrad^a_ij      (Eq. 13),
 * with Qgrad^a_ij = <phi_i|grad|phi_j> - <phi~_i|grad|phi~_j> of Eq. 14 given
 * atom after atom as [3][ni][ni] complex blocks (x, y, z), host memory; pass
 * natoms = 0 and Qgrad = NULL without PAW.  v_0 becomes 4 pi (the |q|^2 of v
 * and of |n_0|^2 cancel), so chi0 and E_c of iq include the head and wings.
 * qdir = NULL switches the limit off again (n(0) and v_0 = 0 of q = 0).  The
 * setting lasts until rpa_set_qpoint replaces iq.  rpa_energy_backward
 * differentiates through the head: the G = 0 part of dE/dn flows back through
 * the dipole matrix of Eq. 13 into dE/dC and dE/dP (FP64). */
rpa_status rpa_set_optical(rpa_ctx* ctx, int32_t iq, const double* qdir, int32_t natoms,
                           const int32_t* nproj, const double* Qgrad);

/* Symmetrised inverse dielectric matrix of the RPA at q-point iq,
 *   eps~^-1_GG'(q, i omega_j) = [(1 - v^1/2 chi0 v^1/2)^-1]_GG',
 * for reuse of chi0 by other many-body kernels (e.g. the screened interaction
 * W = v^1/2 eps~^-1 v^1/2 of GW): chi0 as in rpa_chi0 (with the optical
 * limit if set), the Cholesky factor of the log-det, then L^-H L^-1 in FP64.
 * out[nw][NG][NG] complex (full Hermitian matrix), host or device.
 * RPA_ERR_NOT_HPD as for rpa_energy. */
rpa_status rpa_epsilon_inv(rpa_ctx* ctx, int32_t iq, int32_t nw, const double* omega, double* out);

/* chi0_GG'(q, i omega_j) of q-point iq (Eq. 3 summed as Eq. 17) for nw
 * frequencies omega[nw] (host).  Pairs (n at k, m at k+q) with f_n > f_m
 * enter with the real time-reversal-combined weight
 *   w = s / (Omega N_k) (f_n - f_m) 2 (e_n - e_m) / (w^2 + (e_n - e_m)^2).
 * chi_out[nw][NG][NG] (complex, full Hermitian matrix), host or device. */
rpa_status rpa_chi0(rpa_ctx* ctx, int32_t iq, int32_t nw, const double* omega,
                    double* chi_out);

/* E_c = sum_i wq[i] sum_j W[j] / (2 pi) e_{iqs[i]}(omega_j) (Eqs. 1-2) over
 * nq q-points; e_q(w) = ln det(1 - M) + tr M, M = v^1/2 chi0 v^1/2, by a
 * blocked Cholesky on the device (FP64; float-float trailing updates with FP64
 * pivots in the mixed modes, RPA_TUNE_LOGDET).  *Ec host; terms (nullable,
 * host) receives e_q(omega_j) as terms[nq][nw].  RPA_ERR_NOT_HPD if a
 * Cholesky pivot is not positive. */
rpa_status rpa_energy(rpa_ctx* ctx, int32_t nq, const int32_t* iqs,
                      const double* wq, int32_t nw, const double* omega,
                      const double* W, double* Ec, double* terms);

/* Split form of rpa_energy for batching and CUDA graphs (the paper's point of
 * grouping many small independent pieces of work, Sec. 3.2, taken to whole
 * q-point evaluations).  rpa_set_frequencies stores the nw frequencies on the
 * device (host pointer).  rpa_energy_enqueue queues every kernel of an E_c
 * evaluation over the q-points iqs[nq] on the context's stream and returns
 * without waiting; nothing in it synchronises the host, so it can be captured.
 * rpa_energy_collect waits for that stream and reduces the queued evaluation
 * with the weights wq[nq] and W[nw] (host) into *Ec and terms[nq][nw]
 * (nullable), reporting RPA_ERR_NOT_HPD / RPA_ERR_TIMEOUT as rpa_energy does. */
rpa_status rpa_set_frequencies(rpa_ctx* ctx, int32_t nw, const double* omega);
rpa_status rpa_energy_enqueue(rpa_ctx* ctx, int32_t nq, const int32_t* iqs);
rpa_status rpa_energy_collect(rpa_ctx* ctx, const double* wq, const double* W,
                              double* Ec, double* terms);

/* One CUDA graph holding the E_c evaluations of n contexts (for example many
 * (q, cell) instances of different sizes).  All contexts must have been
 * created with the same caller-provided stream and device and have their
 * frequencies set.  ctx i evaluates nq[i] q-points, listed one context after
 * the other in iqs.  rpa_graph_create runs every evaluation once to size the
 * buffers, then captures them into a graph.  rpa_graph_launch replays it on
 * that stream; afterwards call rpa_energy_collect on each context.  The
 * graph is bound to the contexts' buffers: do not change orbitals, q-points,
 * tuning or frequencies of those contexts while the graph is alive.
 * When every context uses RPA_BF16X2 (RPA_TUNE_BATCH_PERSIST of ctxs[0] = 1,
 * the default), the graph is built around persistent launches: the k-blocks
 * of all contexts and q-points are packed, in order, into groups (at most
 * RPA_TUNE_BATCH_MB, 16 GiB by default, of rank-k operands and 24 blocks
 * each; a larger block alone); per group the pair densities and operand
 * preparation of its blocks run into a graph-owned buffer, one persistent
 * tensor-core launch (one CTA per SM)
 * pulls every (block, tile, frequency) item of the group from a device queue,
 * and the log-dets of the q-points completed by the group follow.  Results
 * are bit-identical to the per-context form.  That buffer and the queue are
 * allocated here and freed by rpa_graph_destroy. */
typedef struct rpa_graph rpa_graph;
rpa_status rpa_graph_create(rpa_ctx* const* ctxs, int32_t n, const int32_t* nq,
                            const int32_t* iqs, rpa_graph** out);
rpa_status rpa_graph_launch(rpa_graph* graph);
void rpa_graph_destroy(rpa_graph* graph);

/* Gradient of E_c (the derivative of Eqs. 1-2 through Eq. 3/17, the PAW term of
 * Eq. 6 and the pair densities of Eqs. 4/10), scaled by dEc.  Same q-points,
 * weights and frequencies as rpa_energy; *Ec (nullable, host) receives E_c.
 * Convention: g = 2 dE/d(conj z), so dE = Re sum conj(g) dz (PyTorch's complex
 * gradient).  For each s < nsets, set_ids[s] names an orbital set and
 *   dC[s] [nbands][npw] complex  receives dE/dC (nullable array or entry),
 *   dP[s] [nbands][sum nproj]    receives dE/dP (nullable; sets without PAW skipped),
 * and dchi[i] (nullable) [nw][NG][NG] complex receives dE/dchi0(q_i, i w_j) =
 * dEc w_q W_j / (2 pi) v^1/2 [1 - (1 - M)^-1] v^1/2.  Band energies and
 * occupations are held fixed.  The pair densities of each (k, k+q) block are
 * recomputed, not stored.  Outputs may be host or device memory.  The
 * (1 - M)^-1 step runs in FP64 on the device (blocked substitution with the
 * Cholesky factor). */
rpa_status rpa_energy_backward(rpa_ctx* ctx, int32_t nq, const int32_t* iqs,
                               const double* wq, int32_t nw, const double* omega,
                               const double* W, double dEc, double* Ec,
                               int32_t nsets, const int32_t* set_ids,
                               double* const* dC, double* const* dP,
                               double* const* dchi);

/* Per-stage device timings of the most recent rpa_chi0/rpa_energy call,
 * measured with CUDA events on the context's stream when enabled by
 * rpa_set_profiling(ctx, 1); the stages group the steps of Table 1 as the
 * paper's per-step timings (Tables 2-3) do.  Index: 0 wavefunctions to grid
 * (step 3), 1 pair densities (+PAW; steps 5-9), 2 rank-k update kernel
 * (step 11), 3 log-det (step 13), 4 other, 5 rank-k operand preparation
 * (split-bfloat16 modes).  ms[RPA_NSTAGES] total
 * milliseconds per stage, launches[RPA_NSTAGES] kernel launches per stage. */
#define RPA_NSTAGES 6
rpa_status rpa_set_profiling(rpa_ctx* ctx, int32_t enable);
rpa_status rpa_get_profile(const rpa_ctx* ctx, double* ms, int64_t* launches);

/* Tuning knobs (they change launch shapes and rounding, never the quantity
 * computed).  The paper's one knob is Nu, the number of unoccupied states
 * grouped into one update (the multi-u approach of Sec. 3.2, Eq. 17); here
 * every pair of a block of occupied bands enters one rank-k launch, and
 * RPA_TUNE_OPERAND_MB and RPA_TUNE_PAIR_CHUNK set those group sizes:
 * RPA_TUNE_TC_FOLD     units of K accumulated in FP32 tensor memory before
 *                      the partial sum is added to FP32 running sums in
 *                      registers (split-bfloat16 modes), in [1, 2^20];
 *                      default 1.  A unit is 64 K-elements in BF16X2 and 32 in
 *                      BF16X3 (twice the products per element), i.e. twelve
 *                      tensor-core accumulation steps either way.  The tensor
 *                      cores truncate while accumulating, so longer folds
 *                      bias |chi0| low.
 * RPA_TUNE_PAIR_CHUNK  pairs per pair-density launch; 0 = sized automatically
 *                      so the transform intermediates stay in L2.
 * RPA_TUNE_TC_FLUSH    folds between additions of the register running sums
 *                      to the FP64 chi0, in [1, 2^20]; default 256.
 * RPA_TUNE_PD_GRID     0 (default): wavefunctions and pair densities use,
 *                      per axis, a grid on which the transform of Eq. 10 has
 *                      no aliasing for the transitions of the call: the
 *                      smallest one, or with RPA_TUNE_PD_FACT = 1 the one of
 *                      least pair-density work among the next eight sizes
 *                      (a size that factorises can cost less than a smaller
 *                      one), never larger than params.grid; results equal
 *                      the plane-wave sums of Eq. 4 either way.
 *                      1: params.grid.
 * RPA_TUNE_OPERAND_MB  device memory (MiB, >= 16) for the pair densities and
 *                      rank-k operands of one block of occupied bands; larger
 *                      pair sets are processed in several blocks.  Default 6144.
 * RPA_TUNE_TC_PIPE     tensor-core pipeline shape: 0 (default) 64-element K
 *                      stages x 2 in shared memory; 1: 32-element stages x 4.
 * RPA_TUNE_LOGDET      arithmetic of the Cholesky trailing updates in the
 *                      RPA_FP32, RPA_BF16X2 and RPA_BF16X3 modes: 2 (default)
 *                      float-float (the part of the matrix still being
 *                      updated held as pairs of FP32, about 44 significant
 *                      bits; finished columns and pivots FP64) with a
 *                      look-ahead of one panel on a second stream (the next
 *                      panel is factorised beside the rest of the current
 *                      update); 1: the same arithmetic on one stream; 0: FP64.
 *                      All three give the same result to rounding.
 *                      RPA_FP64 always uses FP64 on one stream.
 * RPA_TUNE_PAW_TC      the PAW product of Eq. 6 (sum_kp P_m,kp R_n(kp, G), R
 *                      the factor of each occupied band) in the RPA_BF16X2
 *                      and RPA_BF16X3 modes: 0 (default) on the CUDA cores in
 *                      FP32, 1 on the tensor cores with the mode's bfloat16
 *                      split.  1 is faster for many projectors (slab
 *                      workload, 304 projectors: 6.43 -> 6.08 s per q) but
 *                      adds the truncation bias of the tensor cores'
 *                      accumulation to the PAW part of every pair density
 *                      (bulk workload, 39 projectors: E_c within 6.7e-7 of
 *                      FP64 instead of 2.6e-7).  Other modes ignore it.
 * RPA_TUNE_TC_FUSE     RPA_BF16X2 with RPA_TUNE_TC_PIPE = 0: 0 (default)
 *                      stores weighted bfloat16 operands for every frequency
 *                      before the tensor-core kernel; 1 applies the frequency
 *                      weights w_p(w) of Eq. 16 inside the kernel (one
 *                      frequency-independent FP32 copy of the pair densities
 *                      is staged, converter warps scale and split it in
 *                      shared memory): 6x less operand memory and DRAM
 *                      traffic, but the kernel is ~27% slower on GB300 (the
 *                      conversion's shared-memory traffic competes with the
 *                      tensor cores' operand reads).  Both give bit-identical
 *                      chi0.
 * RPA_TUNE_TC_WAIT_US  limit, in microseconds, of every wait of the
 *                      tensor-core kernel on another role's progress, in
 *                      [1000, 60000000]; default 4000000 (4 s).  A wait that
 *                      runs out makes the call return RPA_ERR_TIMEOUT; the
 *                      kernel first lets every load and product it issued
 *                      finish, so the context stays usable.
 * RPA_TUNE_TC_STALL    test of that path: 0 (default) off; k >= 1 makes the
 *                      load role of every tensor-core CTA withhold its K
 *                      stage k-1 and all later ones, so the waits run out.
 * RPA_TUNE_PD_FUSE     0 (default): the middle- and fastest-axis transforms
 *                      of the pair densities run as two kernels through
 *                      global memory; 1: as one kernel per (pair, slab of
 *                      first-axis outputs) through shared memory when a slab
 *                      fits (48 KB), measured 8% slower on the bulk
 *                      workload.  Bit-identical results.
 * RPA_TUNE_BATCH_PERSIST  read from the first context of rpa_graph_create:
 *                      1 (default) builds the graph of a batch whose
 *                      contexts all use RPA_BF16X2 (same RPA_TUNE_TC_FUSE,
 *                      RPA_TUNE_TC_PIPE = 0) around one persistent rank-k
 *                      launch per group of k-blocks (one CTA per SM pulling
 *                      (block, tile, frequency) items of every instance from
 *                      a device queue); 0 captures each context's own
 *                      sequence of launches.  Bit-identical results.
 * RPA_TUNE_BATCH_MB    read from the first context of rpa_graph_create: the
 *                      rank-k operand memory (MiB) of one group of that
 *                      persistent form; default 16384.  An upper bound: where
 *                      the pool cannot be allocated, rpa_graph_create halves
 *                      it (down to the largest single k-block) and re-plans.
 * RPA_TUNE_GAMMA      dE/dchi0 = c_w v^1/2 [1 - (1 - M)^-1] v^1/2 of
 *                      rpa_energy_backward in RPA_FP32, RPA_BF16X2 and
 *                      RPA_BF16X3 (RPA_FP64 always uses FP64): 0 from the
 *                      Cholesky factor in FP64; 2 (default) the same products
 *                      in float-float on the FP32 pipe (about 44 bits; the
 *                      gradient error of the FP64 form); 1 the
 *                      FP32 form -c_w v^1/2 M (1 - M)^-1 v^1/2, fastest but
 *                      with ~1e-5 relative error in dE/dchi0 and ~3e-4 in
 *                      dE/dC and dE/dP on the bulk gradient workload (FP64:
 *                      <= 3e-6).
 * RPA_TUNE_TC_PAIR    the stored-operand two-term rank-k kernel (RPA_BF16X2
 *                      with RPA_TUNE_TC_FUSE = 0 and RPA_TUNE_TC_PIPE = 0):
 *                      0 one CTA per tile; 1 clusters of two CTAs, one tile
 *                      at two frequencies, sharing the unweighted operand
 *                      tiles by TMA multicast (an odd number of frequencies
 *                      runs unpaired); 2 two-SM products (tcgen05
 *                      cta_group::2, M = 256) over pairs of row tiles, each
 *                      SM staging half of the unweighted operand.  All three
 *                      give the same chi0 bit for bit.
 * RPA_TUNE_PD_FACT    1 (default): the slowest and middle axes of the pair
 *                      densities (Eq. 10) as two-level pruned DFTs, the axis
 *                      N = (N / L) L with L in {3, 4, 5, 6, 8} (fewer complex
 *                      multiply-adds per line where that saves a fifth or
 *                      more, at most 16 outputs a line); 0: direct sums.
 *                      The two agree to FP32 rounding.
 * RPA_TUNE_LD_OVERLAP 1 (default): in rpa_energy / rpa_energy_enqueue with
 *                      several q-points, the log-det of one q-point runs on
 *                      a stream of its own beside chi0 of the next (same
 *                      results); 0: one after the other on the context
 *                      stream.
 * Out-of-range values return RPA_ERR_ARG and leave the setting unchanged. */
typedef enum {
  RPA_TUNE_TC_FOLD = 0,
  RPA_TUNE_PAIR_CHUNK = 1,
  RPA_TUNE_TC_FLUSH = 2,
  RPA_TUNE_PD_GRID = 3,
  RPA_TUNE_OPERAND_MB = 4,
  RPA_TUNE_TC_PIPE = 5,
  RPA_TUNE_LOGDET = 6,
  RPA_TUNE_PAW_TC = 7,
  RPA_TUNE_TC_FUSE = 8,
  RPA_TUNE_TC_WAIT_US = 9,
  RPA_TUNE_TC_STALL = 10,
  RPA_TUNE_PD_FUSE = 11,
  RPA_TUNE_BATCH_PERSIST = 12,
  RPA_TUNE_BATCH_MB = 13,
  RPA_TUNE_GAMMA = 14,
  RPA_TUNE_TC_PAIR = 15,
  RPA_TUNE_PD_FACT = 16,
  RPA_TUNE_LD_OVERLAP = 17,
  RPA_TUNE_COUNT = 18
} rpa_tuning;
rpa_status rpa_set_tuning(rpa_ctx* ctx, int32_t param, int64_t value);

/* Allocation-free log-det terms, for callers that must not allocate device
 * memory themselves: code whose device memory is owned by another allocator
 * (a framework's caching pool, or a fixed per-process budget) and loops that
 * cannot afford cudaMalloc/cudaFree, which may synchronize the device.  The
 * paper has no counterpart; this is the FP64 log-det of the energy path
 * (rpa_energy) made callable on its own without a context.
 *
 * For each frequency w < nw it writes
 *   terms[w] = ln det(1 - v^1/2 chi[w] v^1/2) + tr(v^1/2 chi[w] v^1/2)
 * chi: device [nw][ng][ng] complex (interleaved doubles; only the lower
 * triangle is read), v: device [ng], terms: device [nw].  The work runs on
 * `stream` (a cudaStream_t; NULL = the legacy default stream) of the current
 * device, and the call returns after that stream has finished it.
 *
 * Scratch: one process-wide static device array per device (17 MiB + 1040 B,
 * held until the process exits).  Limits: 1 <= nw <= 64 and
 * nw * ng * ng <= 1048576 (e.g. ng <= 256 at nw = 16); larger sizes, null or
 * host pointers, and device memory of a GPU other than the current device
 * return RPA_ERR_ARG without touching the GPU.  The first call on
 * a device looks up the scratch address on that device (cudaGetSymbolAddress);
 * make that first call before any stream capture.  It calls no cudaMalloc,
 * cudaFree or other allocating routine.  Every call reuses the same array and
 * leaves its contents behind (each call rewrites what it reads), so calls
 * that overlap on the GPU, from several host threads or several streams, race
 * and must be serialised by the caller.  Returns RPA_ERR_NOT_HPD if a Cholesky
 * pivot is not positive, RPA_ERR_CUDA on a CUDA error. */
rpa_status rpa_logdet_noalloc(const double* chi, const double* v, int32_t nw,
                              int32_t ng, double* terms, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RPA_GB300_H */
