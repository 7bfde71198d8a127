// Host runtime of the C ABI declared in include/rpa.h: context, argument
// validation, device memory, and the orchestration of the hot path
//   wavefunctions -> grid (Eq. 8), pair densities + PAW (Eqs. 4, 6, 10),
//   grouped rank-k update (Eq. 17), log-det + quadrature (Eqs. 1-2).
// Every arithmetic step runs in the CUDA kernels; the host only builds index
// lists (G spheres, Miller boxes, pair selections) and launches.
#include "rpa.h"
#include "rpa_internal.h"

#include <algorithm>
#include <cmath>
#include <array>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <map>
#include <string>
#include <vector>

namespace rpa {
// tensor-core rank-k update (k_herk_tc.cu): operand preparation (bf16 split of
// the weighted and plain pair densities into scratch), then the tcgen05 kernel
cudaError_t herk_tc_prepare(const float2* N, int64_t P, int NG, const float* wgt, int nw, int split_terms, int fused,
                            void* scratch, size_t scratch_bytes, cudaStream_t s);
cudaError_t herk_tc_run(int64_t P, int NG, int nw, int split_terms, int fused, int fold_stages, int flush_folds, int pipe,
                        int pair, int64_t wait_us, int stall_stage, double2* chi, void* scratch, size_t scratch_bytes,
                        int* err, cudaStream_t s);
size_t herk_tc_scratch_bytes(int64_t P, int NG, int nw, int split_terms, int fused);
// persistent launch of many two-term k-blocks (k_herk_tc.cu)
int herk_tc_batch_max_jobs();
cudaError_t herk_tc_batch_run(int njobs, const int64_t* P, const int* NG, const int* nw, void* const* scratch,
                              const size_t* scratch_bytes, const int* unit_of, double2* const* chi, int fused,
                              int fold_stages, int flush_folds, int64_t wait_us, int* queue, int* err,
                              cudaStream_t s);
cudaError_t launch_or_flags(const int* src, int* const* dst, int n, cudaStream_t s);
// adjoint product 2 sum_w w N conj(Gam_w) on the tensor cores (k_herk_tc.cu)
size_t nbar_tc_gam_bytes(int NG, int nw, int terms);
size_t nbar_tc_a_bytes(int64_t P, int NG, int terms);
cudaError_t nbar_tc_prepare_gam(const float2* Gam, int NG, int nw, int terms, void* gbuf, cudaStream_t s);
cudaError_t nbar_tc_run(const float2* N, const float* wgt, int64_t P, int NG, int nw, int terms, const void* gbuf,
                        void* abuf, size_t abytes, float2* out, int* err, cudaStream_t s);
// PAW term N[(y nR + b)][g] += sum_kp Pm[b][kp] R[y][kp][g] on the tensor cores (k_herk_tc.cu)
size_t paw_tc_bytes(int nL, int nR, int KP, int NG, int terms);
cudaError_t paw_tc_run(const float2* Pm, const float2* R, int KP, int nL, int nR, int NG, int terms, void* scratch,
                       size_t bytes, float2* N, int* err, cudaStream_t s);
// adjoint kernels (k_adjoint.cu)
cudaError_t run_gamma(const double2* L, const double* v, const double* cw, int nw, int n, double2* Y, double2* Wm,
                      double2* G64, float2* G32, cudaStream_t s, int64_t* launches);
cudaError_t run_gamma_mixed(const double2* L, const double2* chi, const double* v, const double* cw, int nw, int n,
                            double2* Yb, double2* Wb, double2* G64, float2* G32, cudaStream_t s, int64_t* launches);
cudaError_t run_gamma_ff(const double2* L, const double* v, const double* cw, int nw, int n, double2* Y, double2* Wm,
                         double2* G64, float2* G32, cudaStream_t s, int64_t* launches);
template <typename T>
cudaError_t launch_nbar(const c2<T>* N, int64_t P, int NG, const T* wgt, const c2<T>* Gam, int nw, c2<T>* Nbar,
                        cudaStream_t s);
template <typename T>
cudaError_t launch_paw_adjoint(const c2<T>* Nbar, const c2<T>* R, const c2<T>* Pm, int nL, int nR, int NG, int KP,
                               const double2* Q, const int* atom_of_kp, const int* idx_in_atom, const int* atom_off,
                               const int64_t* q_off, const int* nproj, const int* Lidx, const int* Ridx, c2<T>* Ywork,
                               double2* part, double2* gPk, double2* gPkp, cudaStream_t s);
template <typename T>
cudaError_t launch_adj_stageC(const c2<T>* Nbar, int NG, int64_t p0, int np, int mc, int nR, int ncol, int N3,
                              const int* col_start, const int* col_g, const int* col_g3, double inv_nr,
                              const c2<T>* tw3, c2<T>* T2, cudaStream_t s);
template <typename T>
size_t adj_stageA_fused_smem(int N1, int n1, int A);
int adj_stageA_fused_slices(int mc, int N23);
template <typename T>
cudaError_t launch_adj_stageA_fused(const c2<T>* T1, int A, int mc, int n1, int N1, int N23, const c2<T>* tw,
                                    const c2<T>* Un0, const c2<T>* Un1, const c2<T>* Ukp, const int* Ridx, int m0,
                                    c2<T>* Ubar_kp, c2<T>* Ubar_n0, c2<T>* Ubar_n1, c2<T>* part, cudaStream_t s);
template <typename T>
cudaError_t launch_adj_stageA(const c2<T>* T1, int np, int n1, int N1, int N23, const c2<T>* tw, const c2<T>* Un,
                              const c2<T>* Ukp, const int* Ridx, int nR, int64_t p0, c2<T>* Ubar_kp, c2<T>* Xbar,
                              cudaStream_t s);
template <typename T>
cudaError_t launch_adj_un(const c2<T>* Xbar, int np, int64_t Nr, const c2<T>* Ukp, const int* Ridx, int nR, int64_t p0,
                          c2<T>* Ubar_n, cudaStream_t s);
template <typename T>
cudaError_t launch_twiddle_adj(c2<T>* tw, int N, int lo, int nin, int chunked, cudaStream_t s);
template <typename T>
cudaError_t launch_gather_box(const c2<T>* box, int nb, int npw, const int* pos, int64_t boxsz, double2* dC,
                              cudaStream_t s);
}

using namespace rpa;

namespace {

constexpr int kMaxIndex = 4096;
// twiddle matrices of the pruned transforms (grid axis x 16 outputs, complex
// double) must fit in shared memory
constexpr int kMaxGrid = 768;
// Miller box searched for a response sphere (a cutoff far beyond any grid the
// transforms accept is an argument error, not an hours-long host loop)
constexpr double kMaxSphereBox = 1u << 28;

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

struct OrbSet {
  bool valid = false;
  double k[3] = {0, 0, 0};
  int nb = 0, npw = 0;
  std::vector<int> miller;
  std::vector<double> eps, f;
  int mlo[3] = {0, 0, 0}, mhi[3] = {0, 0, 0};
  double2* C = nullptr;
  double* eps_d = nullptr;
  double* f_d = nullptr;
  int* pos_d = nullptr;  // flat Miller-box position of each plane wave
  std::vector<int> L, R;  // bands with f > 0 (left of a pair), f < 1 (right)
  int* L_d = nullptr;
  int* R_d = nullptr;
  int natoms = 0;
  std::vector<int> nproj;
  int KP = 0;
  double2* P = nullptr;
  void* U = nullptr;  // grids [nb][Nr] in working precision (valid while grid_stamp == ctx stamp)
  size_t Ubytes = 0;
  uint64_t grid_stamp = 0;
};

struct QPt {
  bool valid = false;
  double q[3] = {0, 0, 0};
  std::vector<int> k_of, kq_of, G0;
  int NG = 0;
  std::vector<int> gm;  // [NG][3]
  std::vector<double> v;
  double* v_d = nullptr;
  int natoms = 0;
  std::vector<int> nproj;
  double2* Q = nullptr;
  int* gfft_d = nullptr;    // [nk][NG][3] transform indices g = G + G0 of every transition
  char* paw_meta_d = nullptr;  // PAW index tables (q offsets, atom of projector, ...)
  int KP = 0;
  // optical limit (Eqs. 12-14), q = 0 only
  bool optical = false;
  int ig0 = -1;                 // index of G = 0 in the sphere
  double2* Qn_d = nullptr;      // q^.Qgrad as a dense block-diagonal [KPo][KPo], or null
  int KPo = 0;
  std::map<int, double*> s_d;   // per orbital set: q^.(k+Q) of its plane waves (made on first use)
  double qhat[3] = {0, 0, 0};   // the normalised direction q^
};


}  // namespace

struct rpa_ctx {
  rpa_params prm{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // second stream of the tensor-core pipeline (operand preparation of the next
  // block beside the rank-k kernel of the current one) and its events
  cudaStream_t stream2 = nullptr;
  cudaEvent_t ev_pd[2] = {nullptr, nullptr}, ev_prep[2] = {nullptr, nullptr}, ev_herk[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // second stream and events of the look-ahead Cholesky (float-float log-det)
  LogdetStreams ld{nullptr, nullptr, nullptr};
  // stream of the log-dets that overlap the next q-point's chi0, and its events
  cudaStream_t ld_stream = nullptr;
  cudaEvent_t ev_chi = nullptr, ev_formed = nullptr, ev_ld = nullptr;
  double B[9] = {0};  // reciprocal rows
  double volume = 0.0;
  std::string err;
  std::map<int, OrbSet> sets;
  std::map<int, QPt> qpts;
  std::map<std::string, DevBuf> ws;
  uint64_t stamp = 0;
  bool profiling = false;
  double prof_ms[RPA_NSTAGES] = {0};
  int64_t prof_launch[RPA_NSTAGES] = {0};
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  int64_t tune[RPA_TUNE_COUNT] = {1, 0, 256, 0, 6144, 0, 2, 0, 0, 4000000, 0, 0, 1, 16384, 2, 0, 1, 1};  // see rpa_tuning in rpa.h
  double* omega_d = nullptr;  // frequencies of rpa_set_frequencies (device)
  int nw_set = 0;
  std::vector<int> enq_iqs;   // q-points of the last rpa_energy_enqueue
  int tg[3] = {0, 0, 0};  // transform grid of the current call (<= prm.grid)
  int* dev_err = nullptr;                 // device-side flag of bounded waits that gave up
};

namespace {

rpa_status fail(rpa_ctx* c, rpa_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return st;
}

#define CUDA_OK(ctx, call)                                                                          \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      if (e_ == cudaErrorMemoryAllocation) return fail(ctx, RPA_ERR_OOM, "%s: %s", #call, cudaGetErrorString(e_)); \
      return fail(ctx, RPA_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));                       \
    }                                                                                               \
  } while (0)

rpa_status dev_alloc(rpa_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return RPA_OK;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, RPA_ERR_OOM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  return RPA_OK;
}

void dev_free(void* p) {
  if (p) cudaFree(p);
}
void free_optical(QPt& Q) {
  dev_free(Q.Qn_d);
  Q.Qn_d = nullptr;
  for (auto& kv : Q.s_d) dev_free(kv.second);
  Q.s_d.clear();
  Q.optical = false;
  Q.KPo = 0;
}

// q^.(k+Q) of every plane wave of orbital set id (Cartesian, B rows) for the
// optical limit of Q, uploaded on first use; rpa_set_orbitals drops it when
// the set's plane waves change.
rpa_status optical_s(rpa_ctx* c, QPt& Q, int id, const double** out) {
  auto it = Q.s_d.find(id);
  if (it != Q.s_d.end()) {
    *out = it->second;
    return RPA_OK;
  }
  const OrbSet& os = c->sets[id];
  const double* B = c->B;
  std::vector<double> sv(os.npw);
  for (int g = 0; g < os.npw; ++g) {
    const double r[3] = {os.k[0] + os.miller[3 * g], os.k[1] + os.miller[3 * g + 1], os.k[2] + os.miller[3 * g + 2]};
    double acc = 0.0;
    for (int d = 0; d < 3; ++d) acc += Q.qhat[d] * (r[0] * B[d] + r[1] * B[3 + d] + r[2] * B[6 + d]);
    sv[g] = acc;
  }
  double* sd = nullptr;
  rpa_status st = dev_alloc(c, (void**)&sd, sizeof(double) * os.npw);
  if (st != RPA_OK) return st;
  Q.s_d[id] = sd;
  CUDA_OK(c, cudaMemcpy(sd, sv.data(), sizeof(double) * os.npw, cudaMemcpyHostToDevice));
  *out = sd;
  return RPA_OK;
}

rpa_status workspace(rpa_ctx* c, const char* name, size_t bytes, void** out) {
  DevBuf& b = c->ws[name];
  if (b.cap < bytes) {
    dev_free(b.p);
    b.p = nullptr;
    b.cap = 0;
    size_t want = bytes + bytes / 8;
    rpa_status st = dev_alloc(c, &b.p, want);
    if (st != RPA_OK) return st;
    b.cap = want;
  }
  *out = b.p;
  return RPA_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Arguments the host reads or writes itself (index lists, frequencies,
// weights, small parameter arrays, scalar outputs) must be host-readable:
// device memory there is an argument error, not a crash of the process.
// Pageable, pinned and managed memory qualify; NULL is left to each call's
// own null checks.
bool host_readable(const void* p) {
  if (!p) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type != cudaMemoryTypeDevice;
}

// The query runs with the context's device current, as the call's own work
// does, so it never starts a context on another device.
bool on_device(int device) {
  if (cudaSetDevice(device) == cudaSuccess) return true;
  cudaGetLastError();
  return false;
}

rpa_status host_args(rpa_ctx* c, std::initializer_list<const void*> ps) {
  if (!on_device(c->prm.device)) return fail(c, RPA_ERR_CUDA, "cudaSetDevice(%d) failed", c->prm.device);
  for (const void* p : ps)
    if (!host_readable(p)) return fail(c, RPA_ERR_ARG, "an argument the host reads or writes is device memory");
  return RPA_OK;
}

#define HOST_ARGS(c, ...)                                  \
  do {                                                     \
    const rpa_status hs_ = host_args((c), {__VA_ARGS__});  \
    if (hs_ != RPA_OK) return hs_;                         \
  } while (0)

rpa_status copy_in(rpa_ctx* c, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return RPA_OK;
  const cudaMemcpyKind kind = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CUDA_OK(c, cudaMemcpyAsync(dst, src, bytes, kind, c->stream));
  return RPA_OK;
}

void inv3(const double* m, double* out) {
  const double a = m[0], b = m[1], cc = m[2], d = m[3], e = m[4], f = m[5], g = m[6], h = m[7], i = m[8];
  const double A = e * i - f * h, Bc = -(d * i - f * g), Cc = d * h - e * g;
  const double det = a * A + b * Bc + cc * Cc;
  out[0] = A / det;
  out[3] = Bc / det;
  out[6] = Cc / det;
  out[1] = -(b * i - cc * h) / det;
  out[4] = (a * i - cc * g) / det;
  out[7] = -(a * h - b * g) / det;
  out[2] = (b * f - cc * e) / det;
  out[5] = -(a * f - cc * d) / det;
  out[8] = (a * e - b * d) / det;
}

double det3(const double* a) {
  return a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) + a[2] * (a[3] * a[7] - a[4] * a[6]);
}

// B = 2 pi inv(cell)^T: row i of B is column i of inv(cell), a_i . b_j = 2 pi delta_ij
void reciprocal_basis(const double* cell, double* B) {
  double inv[9];
  inv3(cell, inv);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) B[3 * i + j] = 2.0 * M_PI * inv[3 * j + i];
}

// Response sphere of Sec. 2.1, {G : |q+G|^2/2 <= ecut}, in Miller-lexicographic
// order (first index slowest), and the Coulomb kernel v_G = 4 pi / |q+G|^2
// (0 where q + G = 0).  The Miller box is bounded by |q+G| <= sqrt(2 ecut)
// through the column norms of inv(B), plus a margin of 2 for q.  False if
// that box exceeds kMaxSphereBox points (or ecut is not finite).
bool response_sphere(const double* B, const double* q, double ecut, std::vector<int>& gm, std::vector<double>& v) {
  gm.clear();
  v.clear();
  const double rmax = std::sqrt(2.0 * ecut);
  double Binv[9];
  inv3(B, Binv);
  int ext[3];
  double box = 1.0;
  for (int i = 0; i < 3; ++i) {
    const double colnorm = std::sqrt(Binv[i] * Binv[i] + Binv[3 + i] * Binv[3 + i] + Binv[6 + i] * Binv[6 + i]);
    const double e = std::ceil(rmax * colnorm) + 2.0;
    if (!(e <= kMaxSphereBox)) return false;
    ext[i] = (int)e;
    box *= 2.0 * e + 1.0;
  }
  if (box > kMaxSphereBox) return false;
  for (int g1 = -ext[0]; g1 <= ext[0]; ++g1)
    for (int g2 = -ext[1]; g2 <= ext[1]; ++g2)
      for (int g3 = -ext[2]; g3 <= ext[2]; ++g3) {
        const double r[3] = {g1 + q[0], g2 + q[1], g3 + q[2]};
        double w[3];
        for (int cc = 0; cc < 3; ++cc) w[cc] = r[0] * B[cc] + r[1] * B[3 + cc] + r[2] * B[6 + cc];
        const double k2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
        if (0.5 * k2 <= ecut) {
          gm.push_back(g1);
          gm.push_back(g2);
          gm.push_back(g3);
          v.push_back((r[0] == 0.0 && r[1] == 0.0 && r[2] == 0.0) ? 0.0 : 4.0 * M_PI / k2);
        }
      }
  return true;
}

// ---- profiling helpers (CUDA events on the context stream)
void prof_begin(rpa_ctx* c) {
  for (int i = 0; i < RPA_NSTAGES; ++i) {
    c->prof_ms[i] = 0;
    c->prof_launch[i] = 0;
  }
  c->ev.clear();
  c->ev_used = 0;
}
cudaEvent_t next_event(rpa_ctx* c) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->ev_pool.push_back(e);
  }
  return c->ev_pool[c->ev_used++];
}
struct StageTimer {
  rpa_ctx* c;
  int stage;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  StageTimer(rpa_ctx* cc, int s, int64_t launches, cudaStream_t stream = nullptr)
      : c(cc), stage(s), st(stream ? stream : cc->stream) {
    c->prof_launch[s] += launches;
    if (c->profiling) {
      a = next_event(c);
      cudaEventRecord(a, st);
    }
  }
  void add_launches(int64_t n) { c->prof_launch[stage] += n; }
  ~StageTimer() {
    if (c->profiling) {
      cudaEvent_t b = next_event(c);
      cudaEventRecord(b, st);
      c->ev.push_back({stage, {a, b}});
    }
  }
};
void prof_end(rpa_ctx* c) {
  if (!c->profiling) return;
  cudaStreamSynchronize(c->stream);
  for (auto& e : c->ev) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e.second.first, e.second.second) == cudaSuccess) c->prof_ms[e.first] += ms;
  }
  c->ev.clear();
}

// float-float trailing updates of the log-det in the mixed-precision modes
bool ff_logdet(const rpa_ctx* c) { return c->prm.precision != RPA_FP64 && c->tune[RPA_TUNE_LOGDET] >= 1; }

// The look-ahead streams of the float-float log-det (created on first use), or
// nullptr in *la when the factorisation runs on one stream.
rpa_status logdet_streams(rpa_ctx* c, const LogdetStreams** la) {
  *la = nullptr;
  if (!ff_logdet(c) || c->tune[RPA_TUNE_LOGDET] != 2) return RPA_OK;
  if (!c->ld.ev_t) CUDA_OK(c, cudaEventCreateWithFlags(&c->ld.ev_t, cudaEventDisableTiming));
  if (!c->ld.ev_u) CUDA_OK(c, cudaEventCreateWithFlags(&c->ld.ev_u, cudaEventDisableTiming));
  if (!c->ld.s2) CUDA_OK(c, cudaStreamCreateWithFlags(&c->ld.s2, cudaStreamNonBlocking));
  *la = &c->ld;
  return RPA_OK;
}

// ---- stage a1: every band of a set onto the real-space grid (Eq. 8, Table 1 step 3)
template <typename T>
rpa_status build_grids_T(rpa_ctx* c, OrbSet& s) {
  const int N1 = c->tg[0], N2 = c->tg[1], N3 = c->tg[2];
  const int64_t Nr = (int64_t)N1 * N2 * N3;
  const size_t need = sizeof(c2<T>) * (size_t)s.nb * Nr;
  if (s.U && s.Ubytes < need) {
    dev_free(s.U);
    s.U = nullptr;
    s.Ubytes = 0;
  }
  if (!s.U) {
    rpa_status st = dev_alloc(c, &s.U, need);
    if (st != RPA_OK) return st;
    s.Ubytes = need;
  }
  const int L1 = s.mhi[0] - s.mlo[0] + 1, L2 = s.mhi[1] - s.mlo[1] + 1, L3 = s.mhi[2] - s.mlo[2] + 1;
  const int64_t box = (int64_t)L1 * L2 * L3;
  // process bands in batches so the intermediates stay modest
  const int64_t per_band = box + (int64_t)L1 * L2 * N3 + (int64_t)L1 * N2 * N3;
  int64_t nbat = std::max<int64_t>(1, std::min<int64_t>(s.nb, (int64_t)(256ll << 20) / (per_band * (int64_t)sizeof(c2<T>))));
  void* wsp;
  rpa_status st = workspace(c, "grid_tmp", sizeof(c2<T>) * (size_t)(nbat * per_band), &wsp);
  if (st != RPA_OK) return st;
  c2<T>* bx = (c2<T>*)wsp;
  c2<T>* x1 = bx + nbat * box;
  c2<T>* x2 = x1 + nbat * (int64_t)L1 * L2 * N3;
  StageTimer tm(c, 0, 0);
  for (int64_t b0 = 0; b0 < s.nb; b0 += nbat) {
    const int nbb = (int)std::min<int64_t>(nbat, s.nb - b0);
    CUDA_OK(c, cudaMemsetAsync(bx, 0, sizeof(c2<T>) * (size_t)(nbb * box), c->stream));
    CUDA_OK(c, launch_scatter_box<T>(s.C + b0 * s.npw, nbb, s.npw, s.pos_d, box, bx, c->stream));
    // axis 3 (fastest): Miller m3 -> j3
    CUDA_OK(c, launch_dft_axis<T>(bx, x1, nbb, L1 * L2, L3, N3, 1, N3, s.mlo[2], 0, +1, c->stream));
    // axis 2: m2 -> j2
    CUDA_OK(c, launch_dft_axis<T>(x1, x2, nbb, L1, L2, N2, N3, N2, s.mlo[1], 0, +1, c->stream));
    // axis 1: m1 -> j1, straight into the band's grid
    CUDA_OK(c, launch_dft_axis<T>(x2, (c2<T>*)s.U + b0 * Nr, nbb, 1, L1, N1, N2 * N3, N1, s.mlo[0], 0, +1,
                                  c->stream));
    tm.add_launches(4);
  }
  s.grid_stamp = c->stamp;
  return RPA_OK;
}

rpa_status build_grids(rpa_ctx* c, OrbSet& s) {
  if (s.grid_stamp == c->stamp && s.U) return RPA_OK;
  if (c->prm.precision == RPA_FP64) return build_grids_T<double>(c, s);
  return build_grids_T<float>(c, s);
}

// ---- transform grid of a call
// The product conj(u_nk) u_m,k' has plane-wave components Q_m - Q_n; the
// transform of Eq. 10 evaluated at g = G + G0 equals the plane-wave sum of
// Eq. 4 exactly when no other component is congruent to g modulo N, i.e. when
// max(Q_m) - min(Q_n) - min(g) <= N - 1 and min(Q_m) - max(Q_n) - max(g) >= 1 - N.
// The smallest N per axis that satisfies this for every transition of the
// call (and holds each orbital sphere) gives identical results with fewer grid
// points than the caller's grid, which is the upper bound (rpa_set_qpoint
// checked it).  RPA_TUNE_PD_GRID = 1 keeps the caller's grid instead.
void choose_transform_grid(rpa_ctx* c, const int* iqs, int nq) {
  for (int d = 0; d < 3; ++d) c->tg[d] = 2;
  if (c->tune[RPA_TUNE_PD_GRID] == 1) {
    for (int d = 0; d < 3; ++d) c->tg[d] = c->prm.grid[d];
    return;
  }
  int nout[3] = {1, 1, 1}, ngmax = 1;  // widest G+G0 extent per axis, largest sphere
  for (int i = 0; i < nq; ++i) {
    const QPt& Q = c->qpts[iqs[i]];
    ngmax = std::max(ngmax, Q.NG);
    for (size_t t = 0; t < Q.k_of.size(); ++t) {
      const OrbSet& a = c->sets[Q.k_of[t]];
      const OrbSet& b = c->sets[Q.kq_of[t]];
      for (int d = 0; d < 3; ++d) {
        int glo = 1 << 30, ghi = -(1 << 30);
        for (int g = 0; g < Q.NG; ++g) {
          const int v = Q.gm[3 * g + d] + Q.G0[3 * t + d];
          glo = std::min(glo, v);
          ghi = std::max(ghi, v);
        }
        int need = std::max(b.mhi[d] - a.mlo[d] - glo, ghi + a.mhi[d] - b.mlo[d]) + 1;
        need = std::max(need, std::max(a.mhi[d] - a.mlo[d] + 1, b.mhi[d] - b.mlo[d] + 1));
        c->tg[d] = std::max(c->tg[d], need);
        nout[d] = std::max(nout[d], ghi - glo + 1);
      }
    }
  }
  for (int d = 0; d < 3; ++d) c->tg[d] = std::min(c->tg[d], c->prm.grid[d]);
  if (c->tune[RPA_TUNE_PD_FACT] != 1) return;
  // Any grid at least as large is alias-free too; among the next few sizes
  // take the one with the least pair-density work per pair, counted in complex
  // multiply-adds: the products and loads of stage A (2 per point), the
  // slowest and middle axes (direct N n or factorised N L + (N / L) n per
  // line) and the fastest-axis gather (NG N3).
  auto axis = [](int N, int n) -> int64_t {
    const int L = n <= 16 ? factored_radix(N, n) : 0;
    return L ? (int64_t)N * L + (int64_t)(N / L) * n : (int64_t)N * n;
  };
  int best[3] = {c->tg[0], c->tg[1], c->tg[2]};
  int64_t best_cost = -1;
  for (int N1 = c->tg[0]; N1 <= std::min(c->tg[0] + 8, c->prm.grid[0]); ++N1)
    for (int N2 = c->tg[1]; N2 <= std::min(c->tg[1] + 8, c->prm.grid[1]); ++N2)
      for (int N3 = c->tg[2]; N3 <= std::min(c->tg[2] + 8, c->prm.grid[2]); ++N3) {
        const int64_t cost = 2 * (int64_t)N1 * N2 * N3 + (int64_t)N2 * N3 * axis(N1, nout[0]) +
                             (int64_t)nout[0] * N3 * axis(N2, nout[1]) + (int64_t)ngmax * N3;
        if (best_cost < 0 || cost < best_cost) {
          best_cost = cost;
          best[0] = N1;
          best[1] = N2;
          best[2] = N3;
        }
      }
  for (int d = 0; d < 3; ++d) c->tg[d] = best[d];
}

// ---- stages a2-a4 for one q-point: chi accumulates in FP64 lower triangle
// Everything one (k, k+q) block leaves on the device after its pair densities.
template <typename T>
struct Block {
  OrbSet* sk = nullptr;
  OrbSet* skp = nullptr;
  int nL = 0, nR = 0, NG = 0, N1 = 0, N2 = 0, N3 = 0, n1 = 0, n2 = 0, KP = 0;
  int64_t P = 0, Nr = 0, PC = 0;
  int glo[3] = {0, 0, 0};
  std::vector<int> gfft;
  T* w = nullptr;                    // [nw][P] pair weights
  c2<T>* N = nullptr;                // [P][NG] pair densities
  c2<T>* R = nullptr;                // [nL][KP][NG] PAW factors
  c2<T>* Pm = nullptr;               // [nR][KP]
  c2<T>* T1 = nullptr;               // transform scratch
  c2<T>* T2 = nullptr;
  const c2<T>* tw3 = nullptr;         // [N3] exp(2 pi i t / N3) of the transform grid
  const int64_t* q_off = nullptr;    // PAW metadata (device)
  const int* atom_of = nullptr;
  const int* idx_in = nullptr;
  const int* atom_off = nullptr;
  const int* nproj = nullptr;
  int a0 = 0;                        // first occupied row of this block
  const int* Lsub = nullptr;         // device list of the block's occupied bands
};

// Occupied-band rows [a0, a1) of a transition form one block: the pair
// rectangle is always whole rows x all empty bands, so every kernel sees a
// plain (nL x nR) rectangle.  Rows per block bound the N and operand buffers.
// The fused weighting of the tensor-core update applies (two terms, default
// pipeline shape, not switched off).
bool tc_fused(const rpa_ctx* c) {
  return c->prm.precision == RPA_BF16X2 && c->tune[RPA_TUNE_TC_FUSE] == 1 && c->tune[RPA_TUNE_TC_PIPE] == 0;
}

// herk_tc_run with the context's knobs
cudaError_t run_herk_tc(rpa_ctx* c, int64_t P, int NG, int nw, int terms, double2* chi, void* scr, size_t sb) {
  return herk_tc_run(P, NG, nw, terms, tc_fused(c) ? 1 : 0, (int)c->tune[RPA_TUNE_TC_FOLD],
                     (int)c->tune[RPA_TUNE_TC_FLUSH], (int)c->tune[RPA_TUNE_TC_PIPE], (int)c->tune[RPA_TUNE_TC_PAIR],
                     c->tune[RPA_TUNE_TC_WAIT_US],
                     (int)c->tune[RPA_TUNE_TC_STALL] - 1, chi, scr, sb, c->dev_err, c->stream);
}

int rows_per_block(const rpa_ctx* c, int nL, int nR, int NG, int nw) {
  const int64_t NGpad = (NG + 127) / 128 * 128;
  // tensor-core operands: NGpad * 2P * terms * 2 B * (nw + 2), or with the
  // fused weighting NGpad * 2P * (2 terms * 2 B * 2 + 4 B); pair densities: P * NG * 8-16 B
  const int64_t budget = c->tune[RPA_TUNE_OPERAND_MB] << 20;
  const int64_t terms = c->prm.precision == RPA_BF16X3 ? 3 : 2;
  int64_t pmax = tc_fused(c) ? budget / (NGpad * 24) : budget / (NGpad * 4 * terms * (nw + 2));
  if (c->prm.precision == RPA_FP64 || c->prm.precision == RPA_FP32) pmax = budget / (16 * (int64_t)NG);
  int64_t rows = std::max<int64_t>(1, pmax / std::max(1, nR));
  return (int)std::min<int64_t>(rows, nL);
}

// stages a2-a3 (pair densities + PAW) and the pair weights of rows [a0, a1) of one transition
template <typename T>
rpa_status pairs_block(rpa_ctx* c, QPt& Q, int t, int a0, int a1, const double* omega_d, int nw, Block<T>& B,
                       int slot = 0) {
  OrbSet& sk = c->sets[Q.k_of[t]];
  OrbSet& skp = c->sets[Q.kq_of[t]];
  B.sk = &sk;
  B.skp = &skp;
  const int nL = a1 - a0, nR = (int)skp.R.size();
  const int* Lsub = sk.L_d + a0;
  const int64_t P = (int64_t)nL * nR;
  B.nL = nL;
  B.nR = nR;
  B.P = P;
  B.a0 = a0;
  B.Lsub = Lsub;
  if (P == 0) return RPA_OK;
  const int N1 = c->tg[0], N2 = c->tg[1], N3 = c->tg[2];
  const int64_t Nr = (int64_t)N1 * N2 * N3;
  const int NG = Q.NG;
  B.N1 = N1;
  B.N2 = N2;
  B.N3 = N3;
  B.Nr = Nr;
  B.NG = NG;
  const int* G0 = &Q.G0[3 * t];
  // target Fourier indices g = G + G0 (cached on the device per transition) and their box
  std::vector<int>& gfft = B.gfft;
  gfft.assign(3 * (size_t)NG, 0);
  int glo[3] = {1 << 30, 1 << 30, 1 << 30}, ghi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
  for (int i = 0; i < NG; ++i)
    for (int d = 0; d < 3; ++d) {
      const int g = Q.gm[3 * i + d] + G0[d];
      gfft[3 * i + d] = g;
      glo[d] = std::min(glo[d], g);
      ghi[d] = std::max(ghi[d], g);
    }
  const int n1 = ghi[0] - glo[0] + 1, n2 = ghi[1] - glo[1] + 1;
  B.n1 = n1;
  B.n2 = n2;
  for (int d = 0; d < 3; ++d) B.glo[d] = glo[d];
  void* p_gfft = Q.gfft_d + (size_t)3 * NG * t;
  void *p_d, *p_df, *p_w, *p_N, *p_T1, *p_T2;
  rpa_status st;
  if ((st = workspace(c, "pair_d", sizeof(double) * P, &p_d)) != RPA_OK) return st;
  if ((st = workspace(c, "pair_df", sizeof(double) * P, &p_df)) != RPA_OK) return st;
  // the weights and pair densities of two blocks may be alive at once (slots)
  if ((st = workspace(c, slot ? "pair_w1" : "pair_w", sizeof(T) * P * nw, &p_w)) != RPA_OK) return st;
  if ((st = workspace(c, slot ? "Nmat1" : "Nmat", sizeof(c2<T>) * (size_t)P * NG, &p_N)) != RPA_OK) return st;
  const double pref = c->prm.spin_factor / (c->volume * (double)c->prm.nk_bz);
  {
    StageTimer tm(c, 4, 2);
    CUDA_OK(c, launch_pair_params(sk.eps_d, sk.f_d, skp.eps_d, skp.f_d, Lsub, nL, skp.R_d, nR, (double*)p_d,
                                  (double*)p_df, c->stream));
    CUDA_OK(c, launch_pair_weights((double*)p_d, (double*)p_df, omega_d, nw, P, pref,
                                   sizeof(T) == 8 ? (double*)p_w : nullptr, sizeof(T) == 4 ? (float*)p_w : nullptr,
                                   c->stream));
  }
  // PAW factors (FP64 arithmetic, stored in working precision)
  c2<T>* Rp = nullptr;
  c2<T>* Pm = nullptr;
  int KP = 0;
  const bool paw = Q.Q && sk.P && skp.P && Q.natoms > 0;
  if (paw) {
    if (sk.nproj != Q.nproj || skp.nproj != Q.nproj)
      return fail(c, RPA_ERR_ARG, "PAW projector counts of the orbital sets do not match Q of this q-point");
    KP = sk.KP;
    void *p_R, *p_Pm;
    const char* md = Q.paw_meta_d;
    const int64_t* q_off_d = (const int64_t*)md;
    const int* atom_of_d = (const int*)(md + sizeof(int64_t) * Q.natoms);
    const int* idx_in_d = atom_of_d + KP;
    const int* atom_off_d = idx_in_d + KP;
    const int* nproj_d = atom_off_d + Q.natoms;
    B.q_off = q_off_d;
    B.atom_of = atom_of_d;
    B.idx_in = idx_in_d;
    B.atom_off = atom_off_d;
    B.nproj = nproj_d;
    if ((st = workspace(c, "paw_R", sizeof(c2<T>) * (size_t)nL * KP * NG, &p_R)) != RPA_OK) return st;
    if ((st = workspace(c, "paw_Pm", sizeof(c2<T>) * (size_t)nR * KP, &p_Pm)) != RPA_OK) return st;
    Rp = (c2<T>*)p_R;
    Pm = (c2<T>*)p_Pm;
    StageTimer tm(c, 1, 2);
    CUDA_OK(c, launch_paw_R<T>(sk.P, KP, Lsub, nL, Q.Q, atom_of_d, idx_in_d, atom_off_d, q_off_d, nproj_d, NG, Rp,
                               c->stream));
    CUDA_OK(c, launch_gather_P<T>(skp.P, KP, skp.R_d, nR, Pm, c->stream));
  }
  // pair densities in chunks of pairs (intermediates sized to stay in L2)
  const int64_t N23 = (int64_t)N2 * N3;
  const int64_t per_pair = (int64_t)n1 * N23 + (int64_t)n1 * n2 * N3;
  const int64_t budget = (sizeof(T) == 8 ? 160ll : 96ll) << 20;
  int64_t PC = std::max<int64_t>(32, budget / (per_pair * (int64_t)sizeof(c2<T>)));
  if (c->tune[RPA_TUNE_PAIR_CHUNK] > 0) PC = c->tune[RPA_TUNE_PAIR_CHUNK];
  PC = std::min<int64_t>(PC, P);
  if ((st = workspace(c, "pd_T1", sizeof(c2<T>) * (size_t)(PC * (int64_t)n1 * N23), &p_T1)) != RPA_OK) return st;
  if ((st = workspace(c, "pd_T2", sizeof(c2<T>) * (size_t)(PC * (int64_t)n1 * n2 * N3), &p_T2)) != RPA_OK) return st;
  void *p_twA, *p_twB, *p_tw3 = nullptr;
  const size_t twA_n = (size_t)((n1 + 15) / 16) * N1 * 16, twB_n = (size_t)((n2 + 15) / 16) * N2 * 16;
  if ((st = workspace(c, "twA", sizeof(c2<T>) * twA_n, &p_twA)) != RPA_OK) return st;
  if ((st = workspace(c, "twB", sizeof(c2<T>) * twB_n, &p_twB)) != RPA_OK) return st;
  {
    StageTimer tm(c, 1, 2);
    CUDA_OK(c, launch_twiddle_matrix<T>((c2<T>*)p_twA, N1, glo[0], n1, c->stream));
    CUDA_OK(c, launch_twiddle_matrix<T>((c2<T>*)p_twB, N2, glo[1], n2, c->stream));
    // stages B and C fused when a slab of the middle-axis output fits in
    // shared memory and the sphere is ordered by g1 (Miller order)
    int OB = c->tune[RPA_TUNE_PD_FUSE] == 1 ? pd_stageBC_slab<T>(n1, n2, N2, N3) : 0;
    for (int i = 1; OB > 0 && i < NG; ++i)
      if (gfft[3 * i] < gfft[3 * (i - 1)]) OB = 0;
    // the slowest and middle axes as two-level pruned DFTs where that saves work
    const int LA = c->tune[RPA_TUNE_PD_FACT] == 1 && n1 <= 16 ? factored_radix(N1, n1) : 0;
    const int LB = c->tune[RPA_TUNE_PD_FACT] == 1 && OB == 0 && n2 <= 16 ? factored_radix(N2, n2) : 0;
    void *p_tfA = nullptr, *p_tfB = nullptr;
    if (LA) {
      if ((st = workspace(c, "twfA", sizeof(c2<T>) * (size_t)(LA * LA + (N1 / LA) * 16), &p_tfA)) != RPA_OK) return st;
      CUDA_OK(c, launch_twiddle_factored<T>((c2<T>*)p_tfA, N1, LA, glo[0], n1, c->stream));
    }
    if (LB) {
      if ((st = workspace(c, "twfB", sizeof(c2<T>) * (size_t)(LB * LB + (N2 / LB) * 16), &p_tfB)) != RPA_OK) return st;
      CUDA_OK(c, launch_twiddle_factored<T>((c2<T>*)p_tfB, N2, LB, glo[1], n2, c->stream));
    }
    if ((st = workspace(c, "tw3", sizeof(c2<T>) * (size_t)N3, &p_tw3)) != RPA_OK) return st;
    CUDA_OK(c, launch_twiddle_line<T>((c2<T>*)p_tw3, N3, c->stream));
    void* p_g1s = nullptr;
    if (OB > 0) {
      if ((st = workspace(c, "pd_g1start", sizeof(int) * (size_t)(n1 + 1), &p_g1s)) != RPA_OK) return st;
      CUDA_OK(c, launch_g1start((const int*)p_gfft, NG, glo[0], n1, (int*)p_g1s, c->stream));
    }
    // Chunks: with the split stages, every row of the block times a run of
    // unoccupied bands, rows fastest, so that the threads of neighbouring
    // pairs read the same unoccupied band's grid (read once per chunk rather
    // than once per occupied band); with the fused stages B + C, contiguous
    // pair ranges.
    const int nrow = (OB == 0 && nL >= 2 && PC >= nL) ? nL : 1;
    const int64_t cols = nrow > 1 ? PC / nrow : PC;
    const int64_t span = nrow > 1 ? nR : P;
    for (int64_t p0 = 0; p0 < span; p0 += cols) {
      const int np = (int)(std::min<int64_t>(cols, span - p0) * nrow);
      if (LA)
        CUDA_OK(c, launch_pd_stageA_fact<T>((const c2<T>*)sk.U, (const c2<T>*)skp.U, Nr, N1, (int)N23, Lsub, skp.R_d,
                                            nR, p0, np, nrow, (const c2<T>*)p_tfA, LA, n1, (c2<T>*)p_T1,
                                            c->stream));
      else
        CUDA_OK(c, launch_pd_stageA<T>((const c2<T>*)sk.U, (const c2<T>*)skp.U, Nr, N1, (int)N23, Lsub, skp.R_d, nR,
                                       p0, np, nrow, (const c2<T>*)p_twA, n1, (c2<T>*)p_T1, c->stream));
      if (OB > 0) {
        CUDA_OK(c, launch_pd_stageBC<T>((const c2<T>*)p_T1, np, n1, N2, N3, (const c2<T>*)p_twB, n2,
                                        (const int*)p_gfft, (const int*)p_g1s, OB, NG, glo[0], glo[1],
                                        1.0 / (double)Nr, p0, (c2<T>*)p_N, c->stream));
        tm.add_launches(2);
        continue;
      }
      if (LB)
        CUDA_OK(c, launch_pd_stageB_fact<T>((const c2<T>*)p_T1, (c2<T>*)p_T2, np, n1, N2, N3, (const c2<T>*)p_tfB, LB,
                                            n2, c->stream));
      else
        CUDA_OK(c, launch_pd_stageB<T>((const c2<T>*)p_T1, (c2<T>*)p_T2, np, n1, N2, N3, (const c2<T>*)p_twB, n2,
                                       c->stream));
      CUDA_OK(c, launch_pd_stageC<T>((const c2<T>*)p_T2, np, n1, n2, N3, (const int*)p_gfft, NG, glo[0], glo[1],
                                     1.0 / (double)Nr, p0, nrow, nR, (const c2<T>*)p_tw3, (c2<T>*)p_N,
                                     c->stream));
      tm.add_launches(3);
    }
    if (paw) {
      const int prec = c->prm.precision;
      bool done = false;
      if constexpr (sizeof(T) == 4) {
        if ((prec == RPA_BF16X2 || prec == RPA_BF16X3) && c->tune[RPA_TUNE_PAW_TC] == 1) {
          // split-bfloat16 modes: the PAW product on the tensor cores with the
          // same split as the rank-k update
          const int terms = prec == RPA_BF16X3 ? 3 : 2;
          const size_t pb = paw_tc_bytes(nL, nR, KP, NG, terms);
          void* p_pt;
          if ((st = workspace(c, "paw_tc", pb, &p_pt)) != RPA_OK) return st;
          CUDA_OK(c, paw_tc_run(Pm, Rp, KP, nL, nR, NG, terms, p_pt, pb, (float2*)p_N, c->dev_err, c->stream));
          tm.add_launches(3);
          done = true;
        }
      }
      if (!done) {
        CUDA_OK(c, launch_paw_gemm<T>(Rp, Pm, KP, nL, nR, NG, (c2<T>*)p_N, c->stream));
        tm.add_launches(1);
      }
    }
  }
  if (Q.optical) {
    // optical limit: the G = 0 column from q^.<psi_n|grad|psi_m> (Eqs. 12-13)
    const bool pawo = Q.Qn_d && sk.P;
    if (pawo && sk.KP != Q.KPo)
      return fail(c, RPA_ERR_ARG, "projector count of set %d does not match the optical Qgrad", Q.k_of[t]);
    void* p_y = nullptr;
    const size_t ob = sizeof(double2) * (size_t)optical_scratch_elems(nL, nR, sk.npw, pawo ? Q.KPo : 0);
    if ((st = workspace(c, "optical_scratch", ob, &p_y)) != RPA_OK) return st;
    const double* sd;
    if ((st = optical_s(c, Q, Q.k_of[t], &sd)) != RPA_OK) return st;
    StageTimer tm(c, 1, pawo ? 3 : 2);
    CUDA_OK(c, launch_optical_head<T>(sk.C, sk.npw, sd, pawo ? sk.P : nullptr, Q.KPo, Q.Qn_d,
                                      (double2*)p_y, Lsub, nL, skp.R_d, nR, sk.eps_d, NG, Q.ig0, (c2<T>*)p_N,
                                      c->stream));
  }
  B.w = (T*)p_w;
  B.N = (c2<T>*)p_N;
  B.R = Rp;
  B.Pm = Pm;
  B.KP = KP;
  B.T1 = (c2<T>*)p_T1;
  B.T2 = (c2<T>*)p_T2;
  B.tw3 = (const c2<T>*)p_tw3;
  B.PC = PC;
  return RPA_OK;
}

// stages a2-a4 for one transition: pair densities, then the grouped rank-k update
template <typename T>
rpa_status chi_block(rpa_ctx* c, QPt& Q, int t, const double* omega_d, int nw, double2* chi) {
  const int nL = (int)c->sets[Q.k_of[t]].L.size(), nR = (int)c->sets[Q.kq_of[t]].R.size();
  const int rows = rows_per_block(c, nL, nR, Q.NG, nw);
  for (int a0 = 0; a0 < nL; a0 += rows) {
    Block<T> B;
    rpa_status st = pairs_block<T>(c, Q, t, a0, std::min(nL, a0 + rows), omega_d, nw, B);
    if (st != RPA_OK) return st;
    if (B.P == 0) continue;
    const int prec = c->prm.precision;
    if (prec == RPA_FP64 || prec == RPA_FP32) {
      StageTimer tm(c, 2, 1);
      CUDA_OK(c, launch_herk_simt_w<T>(B.N, B.P, B.NG, B.w, nw, chi, c->stream));
    } else {
      const int terms = prec == RPA_BF16X3 ? 3 : 2;
      void* scr = nullptr;
      const int fused = tc_fused(c) ? 1 : 0;
      const size_t sb = herk_tc_scratch_bytes(B.P, B.NG, nw, terms, fused);
      if (sb && (st = workspace(c, "herk_tc", sb, &scr)) != RPA_OK) return st;
      {
        StageTimer tm(c, 5, fused ? 1 : 2);
        CUDA_OK(c, herk_tc_prepare((const float2*)B.N, B.P, B.NG, (const float*)B.w, nw, terms, fused, scr, sb,
                                   c->stream));
      }
      StageTimer tm(c, 2, 1);
      CUDA_OK(c, run_herk_tc(c, B.P, B.NG, nw, terms, chi, scr, sb));
    }
  }
  return RPA_OK;
}

rpa_status check_q_ready(rpa_ctx* c, int iq) {
  auto it = c->qpts.find(iq);
  if (it == c->qpts.end() || !it->second.valid) return fail(c, RPA_ERR_STATE, "q-point %d not set", iq);
  QPt& Q = it->second;
  for (size_t t = 0; t < Q.k_of.size(); ++t) {
    auto a = c->sets.find(Q.k_of[t]);
    auto b = c->sets.find(Q.kq_of[t]);
    if (a == c->sets.end() || !a->second.valid || b == c->sets.end() || !b->second.valid)
      return fail(c, RPA_ERR_STATE, "q-point %d references an orbital set that is not set", iq);
  }
  return RPA_OK;
}

// chi0 of one q-point, enqueued without any host synchronisation (frequencies
// already on the device); bounded-wait failures land in c->dev_err.
// Split-bfloat16 modes: every block of occupied rows of every transition,
// pipelined over two streams.  On the context stream: pair densities of block
// i, then the rank-k kernel of block i-1; on the second stream: the operand
// preparation of block i, which runs beside that rank-k kernel (it needs few
// registers and little shared memory, and is bound by HBM while the rank-k
// kernel is bound by the tensor cores).  Pair densities, weights and operands
// alternate between two slots; events order every reuse.  The second stream
// is forked from and joined back to the context stream, so the sequence can
// be captured in a CUDA graph.
rpa_status chi_tc_pipeline(rpa_ctx* c, QPt& Q, const double* omega_d, int nw, double2* chi) {
  rpa_status st;
  if (!c->stream2) {
    CUDA_OK(c, cudaStreamCreateWithFlags(&c->stream2, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      CUDA_OK(c, cudaEventCreateWithFlags(&c->ev_pd[i], cudaEventDisableTiming));
      CUDA_OK(c, cudaEventCreateWithFlags(&c->ev_prep[i], cudaEventDisableTiming));
      CUDA_OK(c, cudaEventCreateWithFlags(&c->ev_herk[i], cudaEventDisableTiming));
    }
    CUDA_OK(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    CUDA_OK(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  }
  const int terms = c->prm.precision == RPA_BF16X3 ? 3 : 2;
  const int fused = tc_fused(c) ? 1 : 0;
  struct Pending {
    int64_t P = 0;
    int NG = 0;
    void* scr = nullptr;
    size_t sb = 0;
    int slot = 0;
  };
  std::vector<std::array<int, 3>> blocks;  // (transition, a0, a1)
  for (size_t t = 0; t < Q.k_of.size(); ++t) {
    const int nL = (int)c->sets[Q.k_of[t]].L.size(), nR = (int)c->sets[Q.kq_of[t]].R.size();
    const int rows = rows_per_block(c, nL, nR, Q.NG, nw);
    for (int a0 = 0; a0 < nL; a0 += rows) blocks.push_back({(int)t, a0, std::min(nL, a0 + rows)});
  }
  CUDA_OK(c, cudaEventRecord(c->ev_fork, c->stream));
  CUDA_OK(c, cudaStreamWaitEvent(c->stream2, c->ev_fork, 0));
  bool herk_done[2] = {false, false};
  Pending prev;
  bool have_prev = false;
  auto run_herk = [&](const Pending& b) -> rpa_status {
    CUDA_OK(c, cudaStreamWaitEvent(c->stream, c->ev_prep[b.slot], 0));
    {
      StageTimer tm(c, 2, 1);
      CUDA_OK(c, run_herk_tc(c, b.P, b.NG, nw, terms, chi, b.scr, b.sb));
    }
    CUDA_OK(c, cudaEventRecord(c->ev_herk[b.slot], c->stream));
    herk_done[b.slot] = true;
    return RPA_OK;
  };
  for (size_t i = 0; i < blocks.size(); ++i) {
    const int slot = (int)(i & 1);
    Block<float> B;
    if ((st = pairs_block<float>(c, Q, blocks[i][0], blocks[i][1], blocks[i][2], omega_d, nw, B, slot)) != RPA_OK)
      return st;
    if (B.P > 0) {
      Pending cur;
      cur.P = B.P;
      cur.NG = B.NG;
      cur.slot = slot;
      cur.sb = herk_tc_scratch_bytes(B.P, B.NG, nw, terms, fused);
      if (cur.sb && (st = workspace(c, slot ? "herk_tc1" : "herk_tc", cur.sb, &cur.scr)) != RPA_OK) return st;
      CUDA_OK(c, cudaEventRecord(c->ev_pd[slot], c->stream));
      CUDA_OK(c, cudaStreamWaitEvent(c->stream2, c->ev_pd[slot], 0));
      // the slot's operands were last read by the rank-k kernel two blocks back
      if (herk_done[slot]) CUDA_OK(c, cudaStreamWaitEvent(c->stream2, c->ev_herk[slot], 0));
      {
        StageTimer tm(c, 5, 2, c->stream2);
        CUDA_OK(c, herk_tc_prepare((const float2*)B.N, B.P, B.NG, (const float*)B.w, nw, terms, fused, cur.scr,
                                   cur.sb, c->stream2));
      }
      CUDA_OK(c, cudaEventRecord(c->ev_prep[slot], c->stream2));
      if (have_prev && (st = run_herk(prev)) != RPA_OK) return st;
      prev = cur;
      have_prev = true;
    }
  }
  if (have_prev && (st = run_herk(prev)) != RPA_OK) return st;
  // join the second stream back into the context stream
  CUDA_OK(c, cudaEventRecord(c->ev_join, c->stream2));
  CUDA_OK(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  return RPA_OK;
}

rpa_status build_chi_async(rpa_ctx* c, int iq, int nw, const double* p_om, double2** chi_out) {
  rpa_status st = check_q_ready(c, iq);
  if (st != RPA_OK) return st;
  QPt& Q = c->qpts[iq];
  const int NG = Q.NG;
  void* p_chi;
  if ((st = workspace(c, "chi", sizeof(double2) * (size_t)nw * NG * NG, &p_chi)) != RPA_OK) return st;
  CUDA_OK(c, cudaMemsetAsync(p_chi, 0, sizeof(double2) * (size_t)nw * NG * NG, c->stream));
  for (size_t t = 0; t < Q.k_of.size(); ++t) {
    if ((st = build_grids(c, c->sets[Q.k_of[t]])) != RPA_OK) return st;
    if ((st = build_grids(c, c->sets[Q.kq_of[t]])) != RPA_OK) return st;
  }
  if (c->prm.precision == RPA_BF16X2 || c->prm.precision == RPA_BF16X3) {
    if ((st = chi_tc_pipeline(c, Q, p_om, nw, (double2*)p_chi)) != RPA_OK) return st;
  } else {
    for (size_t t = 0; t < Q.k_of.size(); ++t) {
      if (c->prm.precision == RPA_FP64)
        st = chi_block<double>(c, Q, (int)t, p_om, nw, (double2*)p_chi);
      else
        st = chi_block<float>(c, Q, (int)t, p_om, nw, (double2*)p_chi);
      if (st != RPA_OK) return st;
    }
  }
  *chi_out = (double2*)p_chi;
  return RPA_OK;
}

// all device work of an E_c evaluation: chi0 and log-det terms of every q-point
// into res_ld / res_tr / res_flag; no host synchronisation, so it can be captured
rpa_status energy_enqueue(rpa_ctx* c, int nq, const int* iqs, int nw, const double* omega_d) {
  rpa_status st;
  void *p_ld, *p_tr, *p_fl;
  if ((st = workspace(c, "res_ld", sizeof(double) * (size_t)nq * nw, &p_ld)) != RPA_OK) return st;
  if ((st = workspace(c, "res_tr", sizeof(double) * (size_t)nq * nw, &p_tr)) != RPA_OK) return st;
  if ((st = workspace(c, "res_flag", sizeof(int) * (size_t)nq, &p_fl)) != RPA_OK) return st;
  CUDA_OK(c, cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream));
  // The log-det of q-point i runs on its own stream beside chi0 of q-point
  // i + 1, which may overwrite the chi0 buffer once that log-det has formed
  // its matrix; the buffers are sized for the largest q-point first, so no
  // reallocation waits for the device in between.
  const bool overlap = c->tune[RPA_TUNE_LD_OVERLAP] == 1 && nq > 1;
  if (overlap) {
    int ngmax = 0;
    for (int i = 0; i < nq; ++i) ngmax = std::max(ngmax, c->qpts[iqs[i]].NG);
    void* p;
    if ((st = workspace(c, "chi", sizeof(double2) * (size_t)nw * ngmax * ngmax, &p)) != RPA_OK) return st;
    if ((st = workspace(c, "chol", sizeof(double2) * (size_t)logdet_work_elems(nw, ngmax), &p)) != RPA_OK) return st;
    if (!c->ld_stream) CUDA_OK(c, cudaStreamCreateWithFlags(&c->ld_stream, cudaStreamNonBlocking));
    for (cudaEvent_t* e : {&c->ev_chi, &c->ev_formed, &c->ev_ld})
      if (!*e) CUDA_OK(c, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  for (int i = 0; i < nq; ++i) {
    if (overlap && i > 0) CUDA_OK(c, cudaStreamWaitEvent(c->stream, c->ev_formed, 0));
    double2* chi = nullptr;
    if ((st = build_chi_async(c, iqs[i], nw, omega_d, &chi)) != RPA_OK) return st;
    QPt& Q = c->qpts[iqs[i]];
    void* p_work;
    if ((st = workspace(c, "chol", sizeof(double2) * (size_t)logdet_work_elems(nw, Q.NG), &p_work)) != RPA_OK) return st;
    int64_t nl = 0;
    const LogdetStreams* la;
    if ((st = logdet_streams(c, &la)) != RPA_OK) return st;
    cudaStream_t ls = c->stream;
    if (overlap) {
      CUDA_OK(c, cudaEventRecord(c->ev_chi, c->stream));
      CUDA_OK(c, cudaStreamWaitEvent(c->ld_stream, c->ev_chi, 0));
      ls = c->ld_stream;
    }
    StageTimer tm(c, 3, 0, ls);
    CUDA_OK(c, run_logdet(chi, Q.v_d, nw, Q.NG, (double2*)p_work, (double*)p_ld + (size_t)i * nw,
                          (double*)p_tr + (size_t)i * nw, (int*)p_fl + i, ff_logdet(c), ls, &nl, la,
                          overlap ? c->ev_formed : nullptr));
    tm.add_launches(nl);
  }
  if (overlap) {
    CUDA_OK(c, cudaEventRecord(c->ev_ld, c->ld_stream));
    CUDA_OK(c, cudaStreamWaitEvent(c->stream, c->ev_ld, 0));
  }
  c->enq_iqs.assign(iqs, iqs + nq);
  return RPA_OK;
}

// waits for the enqueued evaluation and reduces it on the host
rpa_status energy_collect(rpa_ctx* c, int nw, const double* wq, const double* W, double* Ec, double* terms) {
  const int nq = (int)c->enq_iqs.size();
  if (nq == 0) return fail(c, RPA_ERR_STATE, "no energy evaluation enqueued");
  std::vector<double> ld((size_t)nq * nw), tr((size_t)nq * nw);
  std::vector<int> flag(nq);
  int derr = 0;
  CUDA_OK(c, cudaMemcpyAsync(ld.data(), c->ws["res_ld"].p, sizeof(double) * ld.size(), cudaMemcpyDeviceToHost,
                             c->stream));
  CUDA_OK(c, cudaMemcpyAsync(tr.data(), c->ws["res_tr"].p, sizeof(double) * tr.size(), cudaMemcpyDeviceToHost,
                             c->stream));
  CUDA_OK(c, cudaMemcpyAsync(flag.data(), c->ws["res_flag"].p, sizeof(int) * nq, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaMemcpyAsync(&derr, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  if (derr) return fail(c, RPA_ERR_TIMEOUT, "a bounded device wait gave up in the tensor-core update (code %d)", derr);
  double E = 0.0;
  for (int i = 0; i < nq; ++i) {
    if (flag[i])
      return fail(c, RPA_ERR_NOT_HPD, "1 - v^1/2 chi0 v^1/2 is not positive definite at q-point %d", c->enq_iqs[i]);
    double eq = 0.0;
    for (int j = 0; j < nw; ++j) {
      const double e = ld[(size_t)i * nw + j] + tr[(size_t)i * nw + j];
      if (terms) terms[(size_t)i * nw + j] = e;
      eq += W[j] * e;
    }
    E += wq[i] * eq / (2.0 * M_PI);
  }
  *Ec = E;
  return RPA_OK;
}

rpa_status build_chi(rpa_ctx* c, int iq, int nw, const double* omega_host, double2** chi_out) {
  rpa_status st = check_q_ready(c, iq);
  if (st != RPA_OK) return st;
  QPt& Q = c->qpts[iq];
  const int NG = Q.NG;
  CUDA_OK(c, cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream));
  void *p_chi, *p_om;
  if ((st = workspace(c, "chi", sizeof(double2) * (size_t)nw * NG * NG, &p_chi)) != RPA_OK) return st;
  if ((st = workspace(c, "omega", sizeof(double) * nw, &p_om)) != RPA_OK) return st;
  CUDA_OK(c, cudaMemcpyAsync(p_om, omega_host, sizeof(double) * nw, cudaMemcpyHostToDevice, c->stream));
  CUDA_OK(c, cudaMemsetAsync(p_chi, 0, sizeof(double2) * (size_t)nw * NG * NG, c->stream));
  for (size_t t = 0; t < Q.k_of.size(); ++t) {
    if ((st = build_grids(c, c->sets[Q.k_of[t]])) != RPA_OK) return st;
    if ((st = build_grids(c, c->sets[Q.kq_of[t]])) != RPA_OK) return st;
  }
  for (size_t t = 0; t < Q.k_of.size(); ++t) {
    if (c->prm.precision == RPA_FP64)
      st = chi_block<double>(c, Q, (int)t, (const double*)p_om, nw, (double2*)p_chi);
    else
      st = chi_block<float>(c, Q, (int)t, (const double*)p_om, nw, (double2*)p_chi);
    if (st != RPA_OK) return st;
  }
  int derr = 0;
  CUDA_OK(c, cudaMemcpyAsync(&derr, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  if (derr) return fail(c, RPA_ERR_TIMEOUT, "a bounded device wait gave up in the tensor-core update (code %d)", derr);
  *chi_out = (double2*)p_chi;
  return RPA_OK;
}

// ---- adjoint of one transition: nbar (Eq. 17 adjoint), PAW adjoint (Eq. 6),
// transposed pair-density transforms with the orbital products (Eq. 10)
struct AdjState {
  std::map<int, void*> ubar;      // per set: dE/du grids [nb][Nr] in working precision
  std::map<int, double2*> gP;     // per set: dE/dP accumulators [nb][KP] (FP64)
  std::map<int, double2*> gCo;    // per set: dE/dC through the optical head [nb][npw] (FP64), if any
};

template <typename T>
rpa_status backward_block(rpa_ctx* c, QPt& Q, int t, int a0, int a1, const double* omega_d, int nw,
                          const c2<T>* Gam, const void* gam_tc, AdjState& A) {
  Block<T> B;
  rpa_status st = pairs_block<T>(c, Q, t, a0, a1, omega_d, nw, B);
  if (st != RPA_OK || B.P == 0) return st;
  OrbSet& sk = *B.sk;
  OrbSet& skp = *B.skp;
  const int NG = B.NG, nL = B.nL, nR = B.nR, n1 = B.n1, n2 = B.n2;
  const int N1 = B.N1, N2 = B.N2, N3 = B.N3;
  const int64_t Nr = B.Nr, N23 = (int64_t)N2 * N3;
  void *p_nbar, *p_y, *p_cols, *p_twa, *p_twb, *p_xbar;
  if ((st = workspace(c, "Nbar", sizeof(c2<T>) * (size_t)B.P * NG, &p_nbar)) != RPA_OK) return st;
  c2<T>* Nbar = (c2<T>*)p_nbar;
  StageTimer tm(c, 4, 0);
  if (gam_tc && sizeof(T) == 4) {
    // split-bfloat16 modes: the product on the tensor cores
    const int terms = c->prm.precision == RPA_BF16X3 ? 3 : 2;
    void* p_a;
    const size_t ab = nbar_tc_a_bytes(B.P, NG, terms);
    if ((st = workspace(c, "nbar_a", ab, &p_a)) != RPA_OK) return st;
    CUDA_OK(c, nbar_tc_run((const float2*)B.N, (const float*)B.w, B.P, NG, nw, terms, gam_tc, p_a, ab,
                           (float2*)Nbar, c->dev_err, c->stream));
    tm.add_launches(2);
  } else {
    CUDA_OK(c, launch_nbar<T>(B.N, B.P, NG, B.w, Gam, nw, Nbar, c->stream));
    tm.add_launches(1);
  }
  if (Q.optical) {
    // the G = 0 column came from the head (Eqs. 12-13): its adjoint runs
    // through the dipole matrix, then that column is cleared for the
    // transform and PAW adjoints below (q = 0: the same set at k and k+q)
    const bool pawo = Q.Qn_d && sk.P;
    void* p_oa;
    const size_t ob = sizeof(double2) * (size_t)optical_adj_scratch_elems(nL, nR, pawo ? Q.KPo : 0);
    if ((st = workspace(c, "optical_adj", ob, &p_oa)) != RPA_OK) return st;
    const double* sd;
    if ((st = optical_s(c, Q, Q.k_of[t], &sd)) != RPA_OK) return st;
    CUDA_OK(c, launch_optical_adjoint<T>(Nbar, NG, Q.ig0, B.Lsub, nL, skp.R_d, nR, sk.eps_d, sk.C, sk.npw,
                                         sd, pawo ? sk.P : nullptr, Q.KPo, Q.Qn_d, (double2*)p_oa,
                                         A.gCo[Q.k_of[t]], A.gP[Q.k_of[t]], c->stream));
    tm.add_launches(pawo ? 7 : 3);
  }
  if (B.KP > 0) {
    void* p_pp;
    if ((st = workspace(c, "paw_y", sizeof(c2<T>) * (size_t)nL * B.KP * NG, &p_y)) != RPA_OK) return st;
    if ((st = workspace(c, "paw_pkp", sizeof(double2) * (size_t)nL * nR * B.KP, &p_pp)) != RPA_OK) return st;
    CUDA_OK(c, launch_paw_adjoint<T>(Nbar, B.R, B.Pm, nL, nR, NG, B.KP, Q.Q, B.atom_of, B.idx_in, B.atom_off,
                                     B.q_off, B.nproj, B.Lsub, skp.R_d, (c2<T>*)p_y, (double2*)p_pp,
                                     A.gP[Q.k_of[t]], A.gP[Q.kq_of[t]], c->stream));
    tm.add_launches(4);
  }
  // sphere points grouped by (g1, g2) column for the transposed fastest-axis transform
  const int ncol = n1 * n2;
  std::vector<int> cstart(ncol + 1, 0), cg(NG), cg3(NG);
  for (int i = 0; i < NG; ++i) ++cstart[1 + (B.gfft[3 * i] - B.glo[0]) * n2 + (B.gfft[3 * i + 1] - B.glo[1])];
  for (int k = 0; k < ncol; ++k) cstart[k + 1] += cstart[k];
  {
    std::vector<int> fill(cstart.begin(), cstart.end() - 1);
    for (int i = 0; i < NG; ++i) {
      const int col = (B.gfft[3 * i] - B.glo[0]) * n2 + (B.gfft[3 * i + 1] - B.glo[1]);
      cg[fill[col]] = i;
      cg3[fill[col]++] = ((B.gfft[3 * i + 2] % N3) + N3) % N3;  // g3 mod N3
    }
  }
  const size_t cbytes = sizeof(int) * (cstart.size() + 2 * (size_t)NG);
  if ((st = workspace(c, "adj_cols", cbytes, &p_cols)) != RPA_OK) return st;
  std::vector<int> cbuf(cstart);
  cbuf.insert(cbuf.end(), cg.begin(), cg.end());
  cbuf.insert(cbuf.end(), cg3.begin(), cg3.end());
  CUDA_OK(c, cudaMemcpyAsync(p_cols, cbuf.data(), cbytes, cudaMemcpyHostToDevice, c->stream));
  const int* col_start = (const int*)p_cols;
  const int* col_g = col_start + ncol + 1;
  const int* col_g3 = col_g + NG;
  if ((st = workspace(c, "tw_adjB", sizeof(c2<T>) * (size_t)((N2 + 15) / 16) * n2 * 16, &p_twb)) != RPA_OK) return st;
  if ((st = workspace(c, "tw_adjA", sizeof(c2<T>) * (size_t)n1 * N1, &p_twa)) != RPA_OK) return st;
  CUDA_OK(c, launch_twiddle_adj<T>((c2<T>*)p_twb, N2, B.glo[1], n2, 1, c->stream));
  CUDA_OK(c, launch_twiddle_adj<T>((c2<T>*)p_twa, N1, B.glo[0], n1, 0, c->stream));
  c2<T>* ub_k = (c2<T>*)A.ubar[Q.k_of[t]];
  c2<T>* ub_kp = (c2<T>*)A.ubar[Q.kq_of[t]];
  const int64_t PCb = std::max<int64_t>(1, std::min<int64_t>(B.PC, nR));
  // Stage A^T fused with both products where it applies (x-bar stays on chip):
  // chunks of two occupied bands x mc unoccupied bands (one ubar_m update
  // for both), else one band; otherwise x-bar through memory, one band per chunk.
  const bool fused = n1 <= 16 && adj_stageA_fused_smem<T>(N1, n1, 1) <= 200 * 1024;
  const int Aw = fused && nL >= 2 && PCb >= 2 && adj_stageA_fused_smem<T>(N1, n1, 2) <= 200 * 1024 ? 2 : 1;
  const int MC = (int)(PCb / Aw);
  if (fused) {
    const size_t pe = (size_t)adj_stageA_fused_slices(MC, (int)N23) * Aw * Nr;
    if ((st = workspace(c, "adj_part", sizeof(c2<T>) * pe, &p_xbar)) != RPA_OK) return st;
  } else if ((st = workspace(c, "Xbar", sizeof(c2<T>) * (size_t)(PCb * Nr), &p_xbar)) != RPA_OK) {
    return st;
  }
  for (int a = 0; a < nL;) {
    const int na = std::min(Aw, nL - a);
    const c2<T>* un0 = (const c2<T>*)sk.U + (int64_t)sk.L[B.a0 + a] * Nr;
    const c2<T>* un1 = (const c2<T>*)sk.U + (int64_t)sk.L[B.a0 + a + na - 1] * Nr;
    for (int m0 = 0; m0 < nR; m0 += MC) {
      const int mc = std::min(MC, nR - m0);
      const int np = na * mc;
      const int64_t p0 = (int64_t)a * nR + m0;
      CUDA_OK(c, launch_adj_stageC<T>(Nbar, NG, p0, np, mc, nR, ncol, N3, col_start, col_g, col_g3,
                                      1.0 / (double)Nr, B.tw3, B.T2, c->stream));
      CUDA_OK(c, launch_pd_stageB<T>(B.T2, B.T1, np, n1, n2, N3, (const c2<T>*)p_twb, N2, c->stream));
      if (fused) {
        CUDA_OK(c, launch_adj_stageA_fused<T>(B.T1, na, mc, n1, N1, (int)N23, (const c2<T>*)p_twa, un0, un1,
                                              (const c2<T>*)skp.U, skp.R_d, m0, ub_kp,
                                              ub_k + (int64_t)sk.L[B.a0 + a] * Nr,
                                              ub_k + (int64_t)sk.L[B.a0 + a + na - 1] * Nr, (c2<T>*)p_xbar,
                                              c->stream));
      } else {
        CUDA_OK(c, launch_adj_stageA<T>(B.T1, np, n1, N1, (int)N23, (const c2<T>*)p_twa, un0, (const c2<T>*)skp.U,
                                        skp.R_d, nR, p0, ub_kp, (c2<T>*)p_xbar, c->stream));
        CUDA_OK(c, launch_adj_un<T>((const c2<T>*)p_xbar, np, Nr, (const c2<T>*)skp.U, skp.R_d, nR, p0,
                                    ub_k + (int64_t)sk.L[B.a0 + a] * Nr, c->stream));
      }
      tm.add_launches(4);
    }
    a += na;
  }
  return RPA_OK;
}

// dE/dC of one set from its dE/du grids: the adjoint of Eq. 8 is the forward
// pruned transform onto the set's Miller box, gathered at its plane waves.
template <typename T>
rpa_status ubar_to_dC(rpa_ctx* c, OrbSet& s, const c2<T>* ub, double2* dC) {
  const int N1 = c->tg[0], N2 = c->tg[1], N3 = c->tg[2];
  const int64_t Nr = (int64_t)N1 * N2 * N3, N23 = (int64_t)N2 * N3;
  const int L1 = s.mhi[0] - s.mlo[0] + 1, L2 = s.mhi[1] - s.mlo[1] + 1, L3 = s.mhi[2] - s.mlo[2] + 1;
  const int64_t box = (int64_t)L1 * L2 * L3;
  const int64_t per_band = (int64_t)L1 * N23 + (int64_t)L1 * L2 * N3 + box;
  const int64_t nbat = std::max<int64_t>(1, std::min<int64_t>(s.nb, (int64_t)(256ll << 20) / (per_band * (int64_t)sizeof(c2<T>))));
  void* wsp;
  rpa_status st = workspace(c, "grid_tmp", sizeof(c2<T>) * (size_t)(nbat * per_band), &wsp);
  if (st != RPA_OK) return st;
  c2<T>* x1 = (c2<T>*)wsp;
  c2<T>* x2 = x1 + nbat * (int64_t)L1 * N23;
  c2<T>* bx = x2 + nbat * (int64_t)L1 * L2 * N3;
  StageTimer tm(c, 4, 0);
  for (int64_t b0 = 0; b0 < s.nb; b0 += nbat) {
    const int nbb = (int)std::min<int64_t>(nbat, s.nb - b0);
    CUDA_OK(c, launch_dft_axis<T>(ub + b0 * Nr, x1, nbb, 1, N1, L1, (int)N23, N1, 0, s.mlo[0], -1, c->stream));
    CUDA_OK(c, launch_dft_axis<T>(x1, x2, nbb, L1, N2, L2, N3, N2, 0, s.mlo[1], -1, c->stream));
    CUDA_OK(c, launch_dft_axis<T>(x2, bx, nbb, L1 * L2, N3, L3, 1, N3, 0, s.mlo[2], -1, c->stream));
    CUDA_OK(c, launch_gather_box<T>(bx, nbb, s.npw, s.pos_d, box, dC + b0 * s.npw, c->stream));
    tm.add_launches(4);
  }
  return RPA_OK;
}

template <typename T>
rpa_status energy_backward_T(rpa_ctx* c, int nq, const int* iqs, const double* wq, int nw, const double* omega,
                             const double* W, double dEc, double* Ec_out, int nsets, const int* set_ids,
                             double* const* dC, double* const* dP, double* const* dchi) {
  rpa_status st;
  // every set a q-point touches needs grids and zeroed adjoint accumulators
  AdjState A;
  std::vector<int> touched;
  for (int i = 0; i < nq; ++i) {
    QPt& Q = c->qpts[iqs[i]];
    for (size_t t = 0; t < Q.k_of.size(); ++t)
      for (int id : {Q.k_of[t], Q.kq_of[t]})
        if (std::find(touched.begin(), touched.end(), id) == touched.end()) touched.push_back(id);
  }
  const int64_t Nr = (int64_t)c->tg[0] * c->tg[1] * c->tg[2];
  bool optical = false;
  for (int i = 0; i < nq; ++i) optical = optical || c->qpts[iqs[i]].optical;
  for (int id : touched) {
    OrbSet& s = c->sets[id];
    if ((st = build_grids(c, s)) != RPA_OK) return st;
    void* p;
    if (optical) {
      const std::string ko = "gCo" + std::to_string(id);
      if ((st = workspace(c, ko.c_str(), sizeof(double2) * (size_t)s.nb * s.npw, &p)) != RPA_OK) return st;
      CUDA_OK(c, cudaMemsetAsync(p, 0, sizeof(double2) * (size_t)s.nb * s.npw, c->stream));
      A.gCo[id] = (double2*)p;
    }
    const std::string key = "ubar" + std::to_string(id);
    if ((st = workspace(c, key.c_str(), sizeof(c2<T>) * (size_t)s.nb * Nr, &p)) != RPA_OK) return st;
    CUDA_OK(c, cudaMemsetAsync(p, 0, sizeof(c2<T>) * (size_t)s.nb * Nr, c->stream));
    A.ubar[id] = p;
    if (s.P) {
      const std::string kp = "gP" + std::to_string(id);
      if ((st = workspace(c, kp.c_str(), sizeof(double2) * (size_t)s.nb * s.KP, &p)) != RPA_OK) return st;
      CUDA_OK(c, cudaMemsetAsync(p, 0, sizeof(double2) * (size_t)s.nb * s.KP, c->stream));
      A.gP[id] = (double2*)p;
    } else {
      A.gP[id] = nullptr;
    }
  }
  double E = 0.0;
  std::vector<double> ld(nw), tr(nw), cw(nw);
  for (int i = 0; i < nq; ++i) {
    double2* chi = nullptr;
    if ((st = build_chi(c, iqs[i], nw, omega, &chi)) != RPA_OK) return st;
    QPt& Q = c->qpts[iqs[i]];
    const int NG = Q.NG;
    const size_t mat = sizeof(double2) * (size_t)nw * NG * NG;
    void *p_work, *p_ld, *p_tr, *p_flag, *p_Y, *p_W, *p_G64, *p_G32 = nullptr, *p_cw;
    if ((st = workspace(c, "chol", sizeof(double2) * (size_t)logdet_work_elems(nw, NG), &p_work)) != RPA_OK) return st;
    if ((st = workspace(c, "logdet", sizeof(double) * nw, &p_ld)) != RPA_OK) return st;
    if ((st = workspace(c, "trace", sizeof(double) * nw, &p_tr)) != RPA_OK) return st;
    if ((st = workspace(c, "flag", sizeof(int), &p_flag)) != RPA_OK) return st;
    if ((st = workspace(c, "adj_Y", mat, &p_Y)) != RPA_OK) return st;
    if ((st = workspace(c, "adj_W", mat, &p_W)) != RPA_OK) return st;
    if ((st = workspace(c, "gamma64", mat, &p_G64)) != RPA_OK) return st;
    if (sizeof(T) == 4 && (st = workspace(c, "gamma32", mat / 2, &p_G32)) != RPA_OK) return st;
    if ((st = workspace(c, "cw", sizeof(double) * nw, &p_cw)) != RPA_OK) return st;
    int64_t nl = 0;
    {
      const LogdetStreams* la;
      if ((st = logdet_streams(c, &la)) != RPA_OK) return st;
      StageTimer tm(c, 3, 0);
      CUDA_OK(c, run_logdet(chi, Q.v_d, nw, NG, (double2*)p_work, (double*)p_ld, (double*)p_tr, (int*)p_flag,
                            ff_logdet(c), c->stream, &nl, la));
      tm.add_launches(nl);
    }
    int flag = 0;
    CUDA_OK(c, cudaMemcpyAsync(ld.data(), p_ld, sizeof(double) * nw, cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(c, cudaMemcpyAsync(tr.data(), p_tr, sizeof(double) * nw, cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(c, cudaMemcpyAsync(&flag, p_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(c, cudaStreamSynchronize(c->stream));
    if (flag) return fail(c, RPA_ERR_NOT_HPD, "1 - v^1/2 chi0 v^1/2 is not positive definite at q-point %d", iqs[i]);
    double eq = 0.0;
    for (int j = 0; j < nw; ++j) {
      eq += W[j] * (ld[j] + tr[j]);
      cw[j] = dEc * wq[i] * W[j] / (2.0 * M_PI);
    }
    E += wq[i] * eq / (2.0 * M_PI);
    CUDA_OK(c, cudaMemcpyAsync(p_cw, cw.data(), sizeof(double) * nw, cudaMemcpyHostToDevice, c->stream));
    nl = 0;
    {
      StageTimer tm(c, 3, 0);
      // (1 - M)^-1: FP64 in the FP64 mode and with RPA_TUNE_GAMMA = 0; in the
      // mixed modes float-float products (2, default) or the FP32 product form (1)
      const int64_t gm = sizeof(T) == 8 ? 0 : c->tune[RPA_TUNE_GAMMA];
      if (gm == 0)
        CUDA_OK(c, run_gamma((const double2*)p_work, Q.v_d, (const double*)p_cw, nw, NG, (double2*)p_Y,
                             (double2*)p_W, (double2*)p_G64, (float2*)p_G32, c->stream, &nl));
      else if (gm == 2)
        CUDA_OK(c, run_gamma_ff((const double2*)p_work, Q.v_d, (const double*)p_cw, nw, NG, (double2*)p_Y,
                                (double2*)p_W, (double2*)p_G64, (float2*)p_G32, c->stream, &nl));
      else
        CUDA_OK(c, run_gamma_mixed((const double2*)p_work, chi, Q.v_d, (const double*)p_cw, nw, NG, (double2*)p_Y,
                                   (double2*)p_W, (double2*)p_G64, (float2*)p_G32, c->stream, &nl));
      tm.add_launches(nl);
    }
    if (dchi && dchi[i]) {
      const bool dev = is_device_ptr(dchi[i]);
      CUDA_OK(c, cudaMemcpyAsync(dchi[i], p_G64, mat, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 c->stream));
    }
    const void* omega_d = nullptr;
    if ((st = workspace(c, "omega", sizeof(double) * nw, (void**)&omega_d)) != RPA_OK) return st;
    const c2<T>* Gam = sizeof(T) == 8 ? (const c2<T>*)p_G64 : (const c2<T>*)p_G32;
    void* gam_tc = nullptr;
    if (c->prm.precision == RPA_BF16X2 || c->prm.precision == RPA_BF16X3) {
      const int terms = c->prm.precision == RPA_BF16X3 ? 3 : 2;
      if ((st = workspace(c, "nbar_gam", nbar_tc_gam_bytes(NG, nw, terms), &gam_tc)) != RPA_OK) return st;
      StageTimer tm(c, 4, nw);
      CUDA_OK(c, nbar_tc_prepare_gam((const float2*)p_G32, NG, nw, terms, gam_tc, c->stream));
    }
    for (size_t t = 0; t < Q.k_of.size(); ++t)
    {
      const int nL = (int)c->sets[Q.k_of[t]].L.size(), nR = (int)c->sets[Q.kq_of[t]].R.size();
      const int rows = rows_per_block(c, nL, nR, NG, nw);
      for (int a0 = 0; a0 < nL; a0 += rows)
        if ((st = backward_block<T>(c, Q, (int)t, a0, std::min(nL, a0 + rows), (const double*)omega_d, nw, Gam,
                                    gam_tc, A)) != RPA_OK)
          return st;
    }
  }
  // gradients with respect to C and P of the requested sets
  for (int s = 0; s < nsets; ++s) {
    const int id = set_ids[s];
    auto it = c->sets.find(id);
    if (it == c->sets.end() || !it->second.valid) return fail(c, RPA_ERR_STATE, "orbital set %d not set", id);
    OrbSet& os = it->second;
    if (dC && dC[s]) {
      void* p;
      if ((st = workspace(c, "dC", sizeof(double2) * (size_t)os.nb * os.npw, &p)) != RPA_OK) return st;
      CUDA_OK(c, cudaMemsetAsync(p, 0, sizeof(double2) * (size_t)os.nb * os.npw, c->stream));
      if (A.ubar.count(id))
        if ((st = ubar_to_dC<T>(c, os, (const c2<T>*)A.ubar[id], (double2*)p)) != RPA_OK) return st;
      if (A.gCo.count(id)) CUDA_OK(c, launch_add_c128((double2*)p, A.gCo[id], (int64_t)os.nb * os.npw, c->stream));
      const bool dev = is_device_ptr(dC[s]);
      CUDA_OK(c, cudaMemcpyAsync(dC[s], p, sizeof(double2) * (size_t)os.nb * os.npw,
                                 dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
      CUDA_OK(c, cudaStreamSynchronize(c->stream));
    }
    if (dP && dP[s] && os.P) {
      const size_t bytes = sizeof(double2) * (size_t)os.nb * os.KP;
      const bool dev = is_device_ptr(dP[s]);
      if (A.gP.count(id) && A.gP[id]) {
        CUDA_OK(c, cudaMemcpyAsync(dP[s], A.gP[id], bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                   c->stream));
      } else if (dev) {
        CUDA_OK(c, cudaMemsetAsync(dP[s], 0, bytes, c->stream));
      } else {
        memset(dP[s], 0, bytes);
      }
    }
  }
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  CUDA_OK(c, cudaGetLastError());
  if (Ec_out) *Ec_out = E;
  return RPA_OK;
}

}  // namespace

// =============================================================== C ABI
extern "C" {

rpa_status rpa_create(const rpa_params* p, rpa_ctx** out) {
  // (no pointer-attribute query here: it would touch the current device
  // before params->device is selected)
  if (!p || !out) return RPA_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < 3; ++i)
    if (p->grid[i] < 2 || p->grid[i] > kMaxGrid) return RPA_ERR_ARG;
  if (!(p->ecut_chi > 0.0) || !(p->spin_factor > 0.0) || p->nk_bz < 1) return RPA_ERR_ARG;
  if (p->precision < RPA_FP64 || p->precision > RPA_BF16X3) return RPA_ERR_ARG;
  const double det = det3(p->cell);
  if (!(std::fabs(det) > 1e-12) || !std::isfinite(det)) return RPA_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || p->device < 0 || p->device >= ndev) {
    cudaGetLastError();
    return RPA_ERR_CUDA;
  }
  if (cudaSetDevice(p->device) != cudaSuccess) return RPA_ERR_CUDA;
  rpa_ctx* c = new rpa_ctx();
  c->prm = *p;
  c->volume = std::fabs(det);
  reciprocal_basis(p->cell, c->B);
  if (p->stream) {
    c->stream = (cudaStream_t)p->stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return RPA_ERR_CUDA;
    }
    c->own_stream = true;
  }
  if (cudaMalloc(&c->dev_err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return RPA_ERR_OOM;
  }
  *out = c;
  return RPA_OK;
}

void rpa_destroy(rpa_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->prm.device);
  cudaStreamSynchronize(c->stream);
  for (auto& kv : c->sets) {
    OrbSet& s = kv.second;
    dev_free(s.C); dev_free(s.eps_d); dev_free(s.f_d); dev_free(s.pos_d);
    dev_free(s.L_d); dev_free(s.R_d); dev_free(s.P); dev_free(s.U);
  }
  for (auto& kv : c->qpts) {
    dev_free(kv.second.v_d);
    dev_free(kv.second.gfft_d);
    dev_free(kv.second.paw_meta_d);
    dev_free(kv.second.Q);
    free_optical(kv.second);
  }
  for (auto& kv : c->ws) dev_free(kv.second.p);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  if (c->stream2) {
    cudaStreamSynchronize(c->stream2);
    for (int i = 0; i < 2; ++i) {
      cudaEventDestroy(c->ev_pd[i]);
      cudaEventDestroy(c->ev_prep[i]);
      cudaEventDestroy(c->ev_herk[i]);
    }
    cudaEventDestroy(c->ev_fork);
    cudaEventDestroy(c->ev_join);
    cudaStreamDestroy(c->stream2);
  }
  if (c->ld.s2) {
    cudaStreamSynchronize(c->ld.s2);
    cudaStreamDestroy(c->ld.s2);
  }
  if (c->ld.ev_t) cudaEventDestroy(c->ld.ev_t);
  if (c->ld.ev_u) cudaEventDestroy(c->ld.ev_u);
  if (c->ld_stream) {
    cudaStreamSynchronize(c->ld_stream);
    cudaStreamDestroy(c->ld_stream);
  }
  for (cudaEvent_t e : {c->ev_chi, c->ev_formed, c->ev_ld})
    if (e) cudaEventDestroy(e);
  dev_free(c->dev_err);
  dev_free(c->omega_d);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* rpa_last_error(const rpa_ctx* c) { return c ? c->err.c_str() : "null context"; }

rpa_status rpa_gauss_legendre(int32_t n, double omega0, double* omega, double* W) {
  if (n < 1 || n > 1024 || !(omega0 > 0.0) || !omega || !W) return RPA_ERR_ARG;
  // Newton iteration on the Legendre polynomial P_n (three-term recurrence),
  // root i started from cos(pi (i + 3/4) / (n + 1/2)); weight 2/((1-x^2) P_n'^2)
  std::vector<double> x(n), w(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  // ascending nodes
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return x[a] < x[b]; });
  for (int i = 0; i < n; ++i) {
    const double z = x[ord[i]];
    omega[i] = omega0 * (1.0 + z) / (1.0 - z);
    W[i] = w[ord[i]] * 2.0 * omega0 / ((1.0 - z) * (1.0 - z));
  }
  return RPA_OK;
}

rpa_status rpa_set_orbitals(rpa_ctx* c, int32_t kidx, const double k_red[3], int32_t nbands, int32_t npw,
                            const int32_t* miller, const double* C, const double* eps, const double* f) {
  if (!c) return RPA_ERR_ARG;
  if (kidx < 0 || kidx >= kMaxIndex) return fail(c, RPA_ERR_ARG, "kidx %d out of range", kidx);
  if (nbands < 1 || npw < 1 || nbands > (1 << 20) || npw > (1 << 24))
    return fail(c, RPA_ERR_ARG, "bad sizes nbands=%d npw=%d", nbands, npw);
  if (!k_red || !miller || !C || !eps || !f) return fail(c, RPA_ERR_ARG, "null pointer argument");
  HOST_ARGS(c, k_red, miller, eps, f);
  CUDA_OK(c, cudaSetDevice(c->prm.device));
  OrbSet s;
  s.valid = true;
  for (int d = 0; d < 3; ++d) s.k[d] = k_red[d];
  s.nb = nbands;
  s.npw = npw;
  s.miller.assign(miller, miller + 3 * (size_t)npw);
  s.eps.assign(eps, eps + nbands);
  s.f.assign(f, f + nbands);
  for (int i = 0; i < nbands; ++i) {
    if (!std::isfinite(s.eps[i])) return fail(c, RPA_ERR_ARG, "eps[%d] not finite", i);
    if (!(s.f[i] >= 0.0 && s.f[i] <= 1.0)) return fail(c, RPA_ERR_ARG, "f[%d] outside [0,1]", i);
    if (s.f[i] > 0.0) s.L.push_back(i);
    if (s.f[i] < 1.0) s.R.push_back(i);
  }
  for (int d = 0; d < 3; ++d) {
    s.mlo[d] = 1 << 30;
    s.mhi[d] = -(1 << 30);
  }
  for (int q = 0; q < npw; ++q)
    for (int d = 0; d < 3; ++d) {
      s.mlo[d] = std::min(s.mlo[d], s.miller[3 * q + d]);
      s.mhi[d] = std::max(s.mhi[d], s.miller[3 * q + d]);
    }
  for (int d = 0; d < 3; ++d)
    if (s.mhi[d] - s.mlo[d] + 1 > c->prm.grid[d])
      return fail(c, RPA_ERR_ARG, "Miller range along axis %d exceeds the grid", d);
  const int L1 = s.mhi[0] - s.mlo[0] + 1, L2 = s.mhi[1] - s.mlo[1] + 1, L3 = s.mhi[2] - s.mlo[2] + 1;
  std::vector<int> pos(npw);
  std::vector<char> seen((size_t)L1 * L2 * L3, 0);
  for (int q = 0; q < npw; ++q) {
    const int i1 = s.miller[3 * q] - s.mlo[0], i2 = s.miller[3 * q + 1] - s.mlo[1], i3 = s.miller[3 * q + 2] - s.mlo[2];
    const size_t flat = ((size_t)i1 * L2 + i2) * L3 + i3;
    if (seen[flat]) return fail(c, RPA_ERR_ARG, "duplicate Miller index at plane wave %d", q);
    seen[flat] = 1;
    pos[q] = (int)flat;
  }
  rpa_status st;
  // A set that replaces one of the same shape (the usual case when the
  // orbitals are updated every step) takes over its device buffers instead of
  // freeing and allocating them again; its grids are marked stale (stamp 0,
  // below every call's stamp) and rebuilt in place by the next call.  The
  // new contents are written on the context stream, after all earlier work
  // that read the buffers (the other streams join the context stream before
  // a call returns), and the upload is complete when this call returns.  If
  // it fails (a CUDA error), the set kidx is dropped rather than kept.
  auto old_it = c->sets.find(kidx);
  {
    // the optical limit's q^.(k+Q) of this set follows its plane waves
    const bool same_pw = old_it != c->sets.end() && old_it->second.miller == s.miller &&
                         old_it->second.k[0] == s.k[0] && old_it->second.k[1] == s.k[1] && old_it->second.k[2] == s.k[2];
    if (!same_pw) {
      bool synced = false;
      for (auto& qp : c->qpts) {
        auto si = qp.second.s_d.find(kidx);
        if (si == qp.second.s_d.end()) continue;
        if (!synced) {
          CUDA_OK(c, cudaStreamSynchronize(c->stream));  // earlier work may still read it
          synced = true;
        }
        dev_free(si->second);
        qp.second.s_d.erase(si);
      }
    }
  }
  if (old_it != c->sets.end()) {
    OrbSet& o = old_it->second;
    if (o.nb == nbands && o.npw == npw) {
      std::swap(s.C, o.C);
      std::swap(s.eps_d, o.eps_d);
      std::swap(s.f_d, o.f_d);
      std::swap(s.pos_d, o.pos_d);
      std::swap(s.U, o.U);
      std::swap(s.Ubytes, o.Ubytes);
      if (o.L.size() == s.L.size()) std::swap(s.L_d, o.L_d);
      if (o.R.size() == s.R.size()) std::swap(s.R_d, o.R_d);
      o.valid = false;  // its buffers now belong to s; dropped below or on failure
    }
  }
  auto cleanup = [&]() {
    dev_free(s.C); dev_free(s.eps_d); dev_free(s.f_d); dev_free(s.pos_d); dev_free(s.L_d); dev_free(s.R_d);
    dev_free(s.U);
    if (old_it != c->sets.end() && !old_it->second.valid) {
      OrbSet& o = old_it->second;
      dev_free(o.C); dev_free(o.eps_d); dev_free(o.f_d); dev_free(o.pos_d);
      dev_free(o.L_d); dev_free(o.R_d); dev_free(o.P); dev_free(o.U);
      c->sets.erase(old_it);
    }
  };
  if (!s.C && (st = dev_alloc(c, (void**)&s.C, sizeof(double2) * (size_t)nbands * npw)) != RPA_OK) { cleanup(); return st; }
  if (!s.eps_d && (st = dev_alloc(c, (void**)&s.eps_d, sizeof(double) * nbands)) != RPA_OK) { cleanup(); return st; }
  if (!s.f_d && (st = dev_alloc(c, (void**)&s.f_d, sizeof(double) * nbands)) != RPA_OK) { cleanup(); return st; }
  if (!s.pos_d && (st = dev_alloc(c, (void**)&s.pos_d, sizeof(int) * npw)) != RPA_OK) { cleanup(); return st; }
  if (!s.L_d && (st = dev_alloc(c, (void**)&s.L_d, sizeof(int) * std::max<size_t>(1, s.L.size()))) != RPA_OK) { cleanup(); return st; }
  if (!s.R_d && (st = dev_alloc(c, (void**)&s.R_d, sizeof(int) * std::max<size_t>(1, s.R.size()))) != RPA_OK) { cleanup(); return st; }
  if ((st = copy_in(c, s.C, C, sizeof(double2) * (size_t)nbands * npw)) != RPA_OK) { cleanup(); return st; }
  cudaError_t ue = cudaSuccess;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (ue == cudaSuccess && bytes) ue = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream);
  };
  up(s.eps_d, s.eps.data(), sizeof(double) * nbands);
  up(s.f_d, s.f.data(), sizeof(double) * nbands);
  up(s.pos_d, pos.data(), sizeof(int) * npw);
  up(s.L_d, s.L.data(), sizeof(int) * s.L.size());
  up(s.R_d, s.R.data(), sizeof(int) * s.R.size());
  if (ue == cudaSuccess) ue = cudaStreamSynchronize(c->stream);
  if (ue != cudaSuccess) {
    cleanup();
    cudaGetLastError();
    return fail(c, RPA_ERR_CUDA, "orbital upload: %s", cudaGetErrorString(ue));
  }
  s.grid_stamp = 0;
  if (old_it != c->sets.end()) {
    OrbSet& o = old_it->second;
    dev_free(o.C); dev_free(o.eps_d); dev_free(o.f_d); dev_free(o.pos_d);
    dev_free(o.L_d); dev_free(o.R_d); dev_free(o.P); dev_free(o.U);
  }
  c->sets[kidx] = s;
  return RPA_OK;
}

rpa_status rpa_set_orbitals_sym(rpa_ctx* c, int32_t kidx, int32_t src, const int32_t* M, const double* tau,
                                int32_t time_reversal, int32_t natoms, const int32_t* atom_map, const double* D) {
  if (!c) return RPA_ERR_ARG;
  if (kidx == src) return fail(c, RPA_ERR_ARG, "target and source set must differ");
  auto it = c->sets.find(src);
  if (it == c->sets.end() || !it->second.valid) return fail(c, RPA_ERR_STATE, "orbital set %d not set", src);
  if (!M) return fail(c, RPA_ERR_ARG, "null rotation");
  HOST_ARGS(c, M, tau, atom_map);
  // M acts on reduced reciprocal coordinates; it must be unimodular and keep
  // lengths: M^T G M = G with the metric G = B B^T of the reciprocal rows
  const int64_t det = (int64_t)M[0] * (M[4] * M[8] - M[5] * M[7]) - (int64_t)M[1] * (M[3] * M[8] - M[5] * M[6]) +
                      (int64_t)M[2] * (M[3] * M[7] - M[4] * M[6]);
  if (det != 1 && det != -1) return fail(c, RPA_ERR_ARG, "rotation matrix is not unimodular");
  double G[9], scale = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0.0;
      for (int d = 0; d < 3; ++d) acc += c->B[3 * i + d] * c->B[3 * j + d];
      G[3 * i + j] = acc;
      scale = std::max(scale, std::fabs(acc));
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) acc += M[3 * a + i] * G[3 * a + b] * M[3 * b + j];
      if (std::fabs(acc - G[3 * i + j]) > 1e-9 * scale)
        return fail(c, RPA_ERR_ARG, "rotation does not preserve the reciprocal metric");
    }
  if (tau && !(std::isfinite(tau[0]) && std::isfinite(tau[1]) && std::isfinite(tau[2])))
    return fail(c, RPA_ERR_ARG, "tau not finite");
  const OrbSet& so = it->second;
  const int sg = time_reversal ? -1 : 1;
  double kr[3], k[3];
  for (int i = 0; i < 3; ++i) {
    kr[i] = M[3 * i] * so.k[0] + M[3 * i + 1] * so.k[1] + M[3 * i + 2] * so.k[2];
    k[i] = sg * kr[i];
  }
  std::vector<int> mil(so.miller.size());
  std::vector<double2> ph(tau ? so.npw : 0);
  for (int q = 0; q < so.npw; ++q) {
    int Qr[3];
    for (int i = 0; i < 3; ++i) {
      Qr[i] = M[3 * i] * so.miller[3 * q] + M[3 * i + 1] * so.miller[3 * q + 1] + M[3 * i + 2] * so.miller[3 * q + 2];
      mil[3 * q + i] = sg * Qr[i];
    }
    if (tau) {
      // exp(-2 pi i (M (k+Q)).tau), before time reversal
      const double x = (kr[0] + Qr[0]) * tau[0] + (kr[1] + Qr[1]) * tau[1] + (kr[2] + Qr[2]) * tau[2];
      const double fr = x - std::nearbyint(x);  // the phase depends on x mod 1
      ph[q] = make_double2(std::cos(2.0 * M_PI * fr), -std::sin(2.0 * M_PI * fr));
    }
  }
  // the source's projections, copied before the new set may replace anything
  const bool paw = so.P && natoms > 0;
  if (so.P && natoms > 0 && natoms != so.natoms)
    return fail(c, RPA_ERR_ARG, "natoms %d does not match the source set's %d", natoms, so.natoms);
  if (paw && (!atom_map || !D)) return fail(c, RPA_ERR_ARG, "atom_map and D are needed for the projections");
  std::vector<int> nproj = so.nproj;
  const int KP = so.KP, nb = so.nb;
  std::vector<int> meta;
  int64_t dtot = 0;
  if (paw) {
    std::vector<int> off(natoms), srcv(natoms), doff(natoms), atom_of(KP), idx_in(KP);
    int o = 0;
    for (int a = 0; a < natoms; ++a) {
      off[a] = o;
      for (int j = 0; j < nproj[a]; ++j) {
        atom_of[o + j] = a;
        idx_in[o + j] = j;
      }
      o += nproj[a];
    }
    for (int a = 0; a < natoms; ++a) {
      if (atom_map[a] < 0 || atom_map[a] >= natoms || nproj[atom_map[a]] != nproj[a])
        return fail(c, RPA_ERR_ARG, "atom_map[%d] = %d invalid", a, atom_map[a]);
      srcv[a] = atom_map[a];
      doff[a] = (int)dtot;
      dtot += (int64_t)nproj[a] * nproj[a];
    }
    meta.insert(meta.end(), off.begin(), off.end());
    meta.insert(meta.end(), srcv.begin(), srcv.end());
    meta.insert(meta.end(), nproj.begin(), nproj.end());
    meta.insert(meta.end(), doff.begin(), doff.end());
    meta.insert(meta.end(), atom_of.begin(), atom_of.end());
    meta.insert(meta.end(), idx_in.begin(), idx_in.end());
  }
  CUDA_OK(c, cudaSetDevice(c->prm.device));
  rpa_status st;
  void *p_meta = nullptr, *p_D = nullptr, *p_P = nullptr;
  if (paw) {
    if ((st = workspace(c, "sym_meta", sizeof(int) * meta.size(), &p_meta)) != RPA_OK) return st;
    if ((st = workspace(c, "sym_D", sizeof(double2) * (size_t)dtot, &p_D)) != RPA_OK) return st;
    if ((st = workspace(c, "sym_P", sizeof(double2) * (size_t)nb * KP, &p_P)) != RPA_OK) return st;
    CUDA_OK(c, cudaMemcpyAsync(p_meta, meta.data(), sizeof(int) * meta.size(), cudaMemcpyHostToDevice, c->stream));
    if ((st = copy_in(c, p_D, D, sizeof(double2) * (size_t)dtot)) != RPA_OK) return st;
    CUDA_OK(c, launch_rotate_P(so.P, nb, KP, natoms, (const int*)p_meta, (const double2*)p_D, time_reversal ? 1 : 0,
                               (double2*)p_P, c->stream));
  }
  // the coefficients travel unchanged to the rotated plane waves (device to device)
  const std::vector<double> eps = so.eps, f = so.f;
  const double2* Csrc = so.C;
  const int npw = so.npw;
  if ((st = rpa_set_orbitals(c, kidx, k, nb, npw, mil.data(), (const double*)Csrc, eps.data(), f.data())) != RPA_OK)
    return st;
  OrbSet& sn = c->sets[kidx];
  if (tau) {
    void* p_ph;
    if ((st = workspace(c, "sym_phase", sizeof(double2) * (size_t)npw, &p_ph)) != RPA_OK) return st;
    CUDA_OK(c, cudaMemcpyAsync(p_ph, ph.data(), sizeof(double2) * (size_t)npw, cudaMemcpyHostToDevice, c->stream));
    CUDA_OK(c, launch_phase(sn.C, nb, npw, (const double2*)p_ph, c->stream));
  }
  if (time_reversal) CUDA_OK(c, launch_conj(sn.C, (int64_t)nb * npw, c->stream));
  if (paw && (st = rpa_set_paw(c, kidx, natoms, nproj.data(), (const double*)p_P)) != RPA_OK) return st;
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  return RPA_OK;
}

rpa_status rpa_set_paw(rpa_ctx* c, int32_t kidx, int32_t natoms, const int32_t* nproj, const double* P) {
  if (!c) return RPA_ERR_ARG;
  auto it = c->sets.find(kidx);
  if (it == c->sets.end() || !it->second.valid) return fail(c, RPA_ERR_STATE, "orbital set %d not set", kidx);
  if (natoms < 1 || natoms > 100000 || !nproj || !P) return fail(c, RPA_ERR_ARG, "bad PAW arguments");
  HOST_ARGS(c, nproj);
  int KP = 0;
  for (int a = 0; a < natoms; ++a) {
    if (nproj[a] < 1 || nproj[a] > 64) return fail(c, RPA_ERR_ARG, "nproj[%d] = %d outside [1,64]", a, nproj[a]);
    KP += nproj[a];
  }
  OrbSet& s = it->second;
  CUDA_OK(c, cudaSetDevice(c->prm.device));
  double2* Pd = nullptr;
  rpa_status st;
  if ((st = dev_alloc(c, (void**)&Pd, sizeof(double2) * (size_t)s.nb * KP)) != RPA_OK) return st;
  if ((st = copy_in(c, Pd, P, sizeof(double2) * (size_t)s.nb * KP)) != RPA_OK) { dev_free(Pd); return st; }
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  dev_free(s.P);
  s.P = Pd;
  s.natoms = natoms;
  s.nproj.assign(nproj, nproj + natoms);
  s.KP = KP;
  return RPA_OK;
}

rpa_status rpa_set_qpoint(rpa_ctx* c, int32_t iq, const double q_red[3], int32_t nk, const int32_t* k_of,
                          const int32_t* kq_of, const int32_t* G0, int32_t* ng_out) {
  if (!c) return RPA_ERR_ARG;
  if (iq < 0 || iq >= kMaxIndex) return fail(c, RPA_ERR_ARG, "iq %d out of range", iq);
  if (!q_red || nk < 1 || nk > kMaxIndex || !k_of || !kq_of || !G0) return fail(c, RPA_ERR_ARG, "bad q-point arguments");
  HOST_ARGS(c, q_red, k_of, kq_of, G0, ng_out);
  QPt Q;
  Q.valid = true;
  for (int d = 0; d < 3; ++d) Q.q[d] = q_red[d];
  Q.k_of.assign(k_of, k_of + nk);
  Q.kq_of.assign(kq_of, kq_of + nk);
  Q.G0.assign(G0, G0 + 3 * (size_t)nk);
  for (int t = 0; t < nk; ++t) {
    for (int which = 0; which < 2; ++which) {
      const int idx = which ? kq_of[t] : k_of[t];
      auto it = c->sets.find(idx);
      if (it == c->sets.end() || !it->second.valid)
        return fail(c, RPA_ERR_STATE, "transition %d references orbital set %d that is not set", t, idx);
    }
  }
  if (!response_sphere(c->B, Q.q, c->prm.ecut_chi, Q.gm, Q.v))
    return fail(c, RPA_ERR_ARG, "response sphere: Miller box over %.0f points (ecut_chi %g)", kMaxSphereBox,
                c->prm.ecut_chi);
  Q.NG = (int)Q.v.size();
  if (Q.NG == 0) return fail(c, RPA_ERR_ARG, "empty response sphere");
  // the Fourier route (Eq. 10) equals the plane-wave sum only without aliasing:
  // every component Q_m - Q_n - (G + G0) must lie strictly inside (-N, N)
  for (int t = 0; t < nk; ++t) {
    const OrbSet& a = c->sets[k_of[t]];
    const OrbSet& b = c->sets[kq_of[t]];
    for (int d = 0; d < 3; ++d) {
      int glo = 1 << 30, ghi = -(1 << 30);
      for (int i = 0; i < Q.NG; ++i) {
        const int g = Q.gm[3 * i + d] + G0[3 * t + d];
        glo = std::min(glo, g);
        ghi = std::max(ghi, g);
      }
      const int hi = b.mhi[d] - a.mlo[d] - glo;
      const int lo = b.mlo[d] - a.mhi[d] - ghi;
      if (hi > c->prm.grid[d] - 1 || lo < -(c->prm.grid[d] - 1))
        return fail(c, RPA_ERR_ARG, "grid axis %d (N=%d) too small: pair-density transform would alias", d,
                    c->prm.grid[d]);
    }
  }
  CUDA_OK(c, cudaSetDevice(c->prm.device));
  rpa_status st;
  if ((st = dev_alloc(c, (void**)&Q.v_d, sizeof(double) * Q.NG)) != RPA_OK) return st;
  CUDA_OK(c, cudaMemcpyAsync(Q.v_d, Q.v.data(), sizeof(double) * Q.NG, cudaMemcpyHostToDevice, c->stream));
  // transform indices g = G + G0 of every transition, kept on the device
  std::vector<int> gfft((size_t)3 * Q.NG * nk);
  for (int t = 0; t < nk; ++t)
    for (int i = 0; i < Q.NG; ++i)
      for (int d = 0; d < 3; ++d) gfft[((size_t)t * Q.NG + i) * 3 + d] = Q.gm[3 * i + d] + G0[3 * t + d];
  if ((st = dev_alloc(c, (void**)&Q.gfft_d, sizeof(int) * gfft.size())) != RPA_OK) {
    dev_free(Q.v_d);
    return st;
  }
  CUDA_OK(c, cudaMemcpyAsync(Q.gfft_d, gfft.data(), sizeof(int) * gfft.size(), cudaMemcpyHostToDevice, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  auto it = c->qpts.find(iq);
  if (it != c->qpts.end()) {
    dev_free(it->second.v_d);
    dev_free(it->second.Q);
    dev_free(it->second.gfft_d);
    dev_free(it->second.paw_meta_d);
    free_optical(it->second);
  }
  c->qpts[iq] = Q;
  if (ng_out) *ng_out = Q.NG;
  return RPA_OK;
}

rpa_status rpa_gvectors(const rpa_ctx* c, int32_t iq, int32_t* ng, int32_t* miller_out) {
  if (!c || !ng) return RPA_ERR_ARG;
  if (!on_device(c->prm.device)) return RPA_ERR_CUDA;
  if (!host_readable(ng) || !host_readable(miller_out)) return RPA_ERR_ARG;
  auto it = c->qpts.find(iq);
  if (it == c->qpts.end() || !it->second.valid) return RPA_ERR_STATE;
  *ng = it->second.NG;
  if (miller_out) memcpy(miller_out, it->second.gm.data(), sizeof(int32_t) * it->second.gm.size());
  return RPA_OK;
}

rpa_status rpa_response_sphere(const double cell[9], const double q_red[3], double ecut_chi, int32_t cap, int32_t* ng,
                               int32_t* miller_out, double* v_out) {
  if (!cell || !q_red || !ng || cap < 0 || !(ecut_chi > 0.0)) return RPA_ERR_ARG;
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(q_red[d])) return RPA_ERR_ARG;
  const double det = det3(cell);
  if (!(std::fabs(det) > 1e-12) || !std::isfinite(det)) return RPA_ERR_ARG;
  double B[9];
  reciprocal_basis(cell, B);
  std::vector<int> gm;
  std::vector<double> v;
  if (!response_sphere(B, q_red, ecut_chi, gm, v)) return RPA_ERR_ARG;
  *ng = (int32_t)v.size();
  if ((miller_out || v_out) && cap < *ng) return RPA_ERR_ARG;
  if (miller_out && !gm.empty()) memcpy(miller_out, gm.data(), sizeof(int32_t) * gm.size());
  if (v_out && !v.empty()) memcpy(v_out, v.data(), sizeof(double) * v.size());
  return RPA_OK;
}

rpa_status rpa_set_optical(rpa_ctx* c, int32_t iq, const double* qdir, int32_t natoms, const int32_t* nproj,
                           const double* Qg) {
  if (!c) return RPA_ERR_ARG;
  HOST_ARGS(c, qdir, nproj, Qg);
  auto it = c->qpts.find(iq);
  if (it == c->qpts.end() || !it->second.valid) return fail(c, RPA_ERR_STATE, "q-point %d not set", iq);
  QPt& Q = it->second;
  CUDA_OK(c, cudaSetDevice(c->prm.device));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));  // earlier work may still read the old tables
  free_optical(Q);
  int ig0 = -1;
  for (int i = 0; i < Q.NG; ++i)
    if (Q.gm[3 * i] == 0 && Q.gm[3 * i + 1] == 0 && Q.gm[3 * i + 2] == 0) ig0 = i;
  if (!qdir) {
    if (ig0 >= 0 && Q.q[0] == 0.0 && Q.q[1] == 0.0 && Q.q[2] == 0.0) {
      Q.v[ig0] = 0.0;
      CUDA_OK(c, cudaMemcpy(Q.v_d + ig0, &Q.v[ig0], sizeof(double), cudaMemcpyHostToDevice));
    }
    return RPA_OK;
  }
  if (Q.q[0] != 0.0 || Q.q[1] != 0.0 || Q.q[2] != 0.0 || ig0 < 0)
    return fail(c, RPA_ERR_ARG, "the optical limit needs q = 0");
  for (size_t t = 0; t < Q.k_of.size(); ++t)
    if (Q.k_of[t] != Q.kq_of[t] || Q.G0[3 * t] || Q.G0[3 * t + 1] || Q.G0[3 * t + 2])
      return fail(c, RPA_ERR_ARG, "the optical limit needs k -> k transitions without umklapp");
  const double nrm = std::sqrt(qdir[0] * qdir[0] + qdir[1] * qdir[1] + qdir[2] * qdir[2]);
  if (!(nrm > 0.0) || !std::isfinite(nrm)) return fail(c, RPA_ERR_ARG, "qdir must be a nonzero vector");
  const double qh[3] = {qdir[0] / nrm, qdir[1] / nrm, qdir[2] / nrm};
  if (natoms < 0 || natoms > 100000 || (natoms > 0 && (!nproj || !Qg)))
    return fail(c, RPA_ERR_ARG, "bad optical PAW arguments");
  rpa_status st;
  if (natoms > 0) {
    int KP = 0;
    for (int a = 0; a < natoms; ++a) {
      if (nproj[a] < 1 || nproj[a] > 64) return fail(c, RPA_ERR_ARG, "nproj[%d] outside [1,64]", a);
      KP += nproj[a];
    }
    if (is_device_ptr(Qg)) return fail(c, RPA_ERR_ARG, "Qgrad must be host memory");
    std::vector<double2> Qn((size_t)KP * KP, make_double2(0.0, 0.0));
    size_t src = 0;
    int off = 0;
    for (int a = 0; a < natoms; ++a) {
      const int ni = nproj[a];
      for (int i = 0; i < ni; ++i)
        for (int j = 0; j < ni; ++j) {
          double2 v = make_double2(0.0, 0.0);
          for (int d = 0; d < 3; ++d) {
            const size_t e = src + ((size_t)d * ni + i) * ni + j;
            v.x += qh[d] * Qg[2 * e];
            v.y += qh[d] * Qg[2 * e + 1];
          }
          Qn[(size_t)(off + i) * KP + off + j] = v;
        }
      src += (size_t)3 * ni * ni;
      off += ni;
    }
    if ((st = dev_alloc(c, (void**)&Q.Qn_d, sizeof(double2) * Qn.size())) != RPA_OK) return st;
    CUDA_OK(c, cudaMemcpy(Q.Qn_d, Qn.data(), sizeof(double2) * Qn.size(), cudaMemcpyHostToDevice));
    Q.KPo = KP;
  }
  // q^.(k+Q) of every plane wave of every set used by iq
  for (int d = 0; d < 3; ++d) Q.qhat[d] = qh[d];
  for (int id : Q.k_of) {
    const double* sd;
    if ((st = optical_s(c, Q, id, &sd)) != RPA_OK) return st;
  }
  Q.ig0 = ig0;
  Q.v[ig0] = 4.0 * M_PI;
  CUDA_OK(c, cudaMemcpy(Q.v_d + ig0, &Q.v[ig0], sizeof(double), cudaMemcpyHostToDevice));
  Q.optical = true;
  return RPA_OK;
}

rpa_status rpa_set_paw_Q(rpa_ctx* c, int32_t iq, int32_t natoms, const int32_t* nproj, const double* Qv) {
  if (!c) return RPA_ERR_ARG;
  auto it = c->qpts.find(iq);
  if (it == c->qpts.end() || !it->second.valid) return fail(c, RPA_ERR_STATE, "q-point %d not set", iq);
  if (natoms < 1 || natoms > 100000 || !nproj || !Qv) return fail(c, RPA_ERR_ARG, "bad PAW Q arguments");
  HOST_ARGS(c, nproj);
  QPt& Q = it->second;
  int64_t tot = 0;
  for (int a = 0; a < natoms; ++a) {
    if (nproj[a] < 1 || nproj[a] > 64) return fail(c, RPA_ERR_ARG, "nproj[%d] outside [1,64]", a);
    tot += (int64_t)nproj[a] * nproj[a] * Q.NG;
  }
  CUDA_OK(c, cudaSetDevice(c->prm.device));
  double2* Qd = nullptr;
  rpa_status st;
  if ((st = dev_alloc(c, (void**)&Qd, sizeof(double2) * (size_t)tot)) != RPA_OK) return st;
  if ((st = copy_in(c, Qd, Qv, sizeof(double2) * (size_t)tot)) != RPA_OK) { dev_free(Qd); return st; }
  // index tables of the projector layout: q offsets per atom, atom and index of
  // every projector, first projector of every atom, projectors per atom
  int KP = 0;
  for (int a = 0; a < natoms; ++a) KP += nproj[a];
  std::vector<int> atom_of(KP), idx_in(KP), atom_off(natoms);
  std::vector<int64_t> q_off(natoms);
  int off = 0;
  int64_t qo = 0;
  for (int a = 0; a < natoms; ++a) {
    atom_off[a] = off;
    q_off[a] = qo;
    for (int j = 0; j < nproj[a]; ++j) {
      atom_of[off + j] = a;
      idx_in[off + j] = j;
    }
    off += nproj[a];
    qo += (int64_t)nproj[a] * nproj[a] * Q.NG;
  }
  const size_t meta_bytes = sizeof(int64_t) * natoms + sizeof(int) * (2 * KP + 2 * natoms);
  std::vector<char> meta(meta_bytes);
  char* mp = meta.data();
  memcpy(mp, q_off.data(), sizeof(int64_t) * natoms);
  mp += sizeof(int64_t) * natoms;
  memcpy(mp, atom_of.data(), sizeof(int) * KP);
  mp += sizeof(int) * KP;
  memcpy(mp, idx_in.data(), sizeof(int) * KP);
  mp += sizeof(int) * KP;
  memcpy(mp, atom_off.data(), sizeof(int) * natoms);
  mp += sizeof(int) * natoms;
  memcpy(mp, nproj, sizeof(int) * natoms);
  char* md = nullptr;
  if ((st = dev_alloc(c, (void**)&md, meta_bytes)) != RPA_OK) {
    dev_free(Qd);
    return st;
  }
  CUDA_OK(c, cudaMemcpyAsync(md, meta.data(), meta_bytes, cudaMemcpyHostToDevice, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  dev_free(Q.Q);
  dev_free(Q.paw_meta_d);
  Q.Q = Qd;
  Q.paw_meta_d = md;
  Q.KP = KP;
  Q.natoms = natoms;
  Q.nproj.assign(nproj, nproj + natoms);
  return RPA_OK;
}

rpa_status rpa_epsilon_inv(rpa_ctx* c, int32_t iq, int32_t nw, const double* omega, double* out) {
  if (!c) return RPA_ERR_ARG;
  if (nw < 1 || nw > 4096 || !omega || !out) return fail(c, RPA_ERR_ARG, "bad rpa_epsilon_inv arguments");
  HOST_ARGS(c, omega);
  CUDA_OK(c, cudaSetDevice(c->prm.device));
  prof_begin(c);
  ++c->stamp;
  rpa_status st = check_q_ready(c, iq);
  if (st != RPA_OK) return st;
  choose_transform_grid(c, &iq, 1);
  double2* chi = nullptr;
  if ((st = build_chi(c, iq, nw, omega, &chi)) != RPA_OK) return st;
  QPt& Q = c->qpts[iq];
  const int NG = Q.NG;
  const size_t mat = sizeof(double2) * (size_t)nw * NG * NG;
  void *p_work, *p_ld, *p_tr, *p_flag, *p_Y, *p_W, *p_cw;
  if ((st = workspace(c, "chol", sizeof(double2) * (size_t)logdet_work_elems(nw, NG), &p_work)) != RPA_OK) return st;
  if ((st = workspace(c, "logdet", sizeof(double) * nw, &p_ld)) != RPA_OK) return st;
  if ((st = workspace(c, "trace", sizeof(double) * nw, &p_tr)) != RPA_OK) return st;
  if ((st = workspace(c, "flag", sizeof(int), &p_flag)) != RPA_OK) return st;
  if ((st = workspace(c, "adj_Y", mat, &p_Y)) != RPA_OK) return st;
  if ((st = workspace(c, "adj_W", mat, &p_W)) != RPA_OK) return st;
  if ((st = workspace(c, "cw", sizeof(double) * nw, &p_cw)) != RPA_OK) return st;
  CUDA_OK(c, cudaMemsetAsync(p_cw, 0, sizeof(double) * nw, c->stream));
  {
    int64_t nl = 0;
    const LogdetStreams* la;
    if ((st = logdet_streams(c, &la)) != RPA_OK) return st;
    StageTimer tm(c, 3, 0);
    CUDA_OK(c, run_logdet(chi, Q.v_d, nw, NG, (double2*)p_work, (double*)p_ld, (double*)p_tr, (int*)p_flag,
                          ff_logdet(c), c->stream, &nl, la));
    // (1 - M)^-1 = L^-H L^-1 from the factor (the Gamma output is not needed)
    CUDA_OK(c, run_gamma((const double2*)p_work, Q.v_d, (const double*)p_cw, nw, NG, (double2*)p_Y, (double2*)p_W,
                         nullptr, nullptr, c->stream, &nl));
    tm.add_launches(nl);
  }
  int flag = 0;
  CUDA_OK(c, cudaMemcpyAsync(&flag, p_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  const bool dev = is_device_ptr(out);
  CUDA_OK(c, cudaMemcpyAsync(out, p_W, mat, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  if (flag) return fail(c, RPA_ERR_NOT_HPD, "1 - v^1/2 chi0 v^1/2 is not positive definite at q-point %d", iq);
  prof_end(c);
  return RPA_OK;
}

rpa_status rpa_chi0(rpa_ctx* c, int32_t iq, int32_t nw, const double* omega, double* chi_out) {
  if (!c) return RPA_ERR_ARG;
  if (nw < 1 || nw > 4096 || !omega || !chi_out) return fail(c, RPA_ERR_ARG, "bad rpa_chi0 arguments");
  HOST_ARGS(c, omega);
  CUDA_OK(c, cudaSetDevice(c->prm.device));
  prof_begin(c);
  ++c->stamp;
  rpa_status st = check_q_ready(c, iq);
  if (st != RPA_OK) return st;
  choose_transform_grid(c, &iq, 1);
  double2* chi = nullptr;
  st = build_chi(c, iq, nw, omega, &chi);
  if (st != RPA_OK) return st;
  const int NG = c->qpts[iq].NG;
  {
    StageTimer tm(c, 4, 1);
    CUDA_OK(c, launch_hermitian_fill(chi, nw, NG, c->stream));
  }
  const size_t bytes = sizeof(double2) * (size_t)nw * NG * NG;
  const bool dev = is_device_ptr(chi_out);
  CUDA_OK(c, cudaMemcpyAsync(chi_out, chi, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  if (!dev || c->profiling) CUDA_OK(c, cudaStreamSynchronize(c->stream));
  CUDA_OK(c, cudaGetLastError());
  prof_end(c);
  return RPA_OK;
}

rpa_status rpa_energy(rpa_ctx* c, int32_t nq, const int32_t* iqs, const double* wq, int32_t nw, const double* omega,
                      const double* W, double* Ec, double* terms) {
  if (!c) return RPA_ERR_ARG;
  if (nq < 1 || nq > kMaxIndex || !iqs || !wq || nw < 1 || nw > 4096 || !omega || !W || !Ec)
    return fail(c, RPA_ERR_ARG, "bad rpa_energy arguments");
  HOST_ARGS(c, iqs, wq, omega, W, Ec, terms);
  CUDA_OK(c, cudaSetDevice(c->prm.device));
  prof_begin(c);
  ++c->stamp;
  for (int i = 0; i < nq; ++i) {
    rpa_status st = check_q_ready(c, iqs[i]);
    if (st != RPA_OK) return st;
  }
  choose_transform_grid(c, iqs, nq);
  void* p_om;
  rpa_status st;
  if ((st = workspace(c, "omega", sizeof(double) * nw, &p_om)) != RPA_OK) return st;
  CUDA_OK(c, cudaMemcpyAsync(p_om, omega, sizeof(double) * nw, cudaMemcpyHostToDevice, c->stream));
  if ((st = energy_enqueue(c, nq, iqs, nw, (const double*)p_om)) != RPA_OK) return st;
  if ((st = energy_collect(c, nw, wq, W, Ec, terms)) != RPA_OK) return st;
  prof_end(c);
  return RPA_OK;
}

rpa_status rpa_set_frequencies(rpa_ctx* c, int32_t nw, const double* omega) {
  if (!c) return RPA_ERR_ARG;
  if (nw < 1 || nw > 4096 || !omega) return fail(c, RPA_ERR_ARG, "bad frequency arguments");
  HOST_ARGS(c, omega);
  for (int j = 0; j < nw; ++j)
    if (!std::isfinite(omega[j])) return fail(c, RPA_ERR_ARG, "omega[%d] not finite", j);
  CUDA_OK(c, cudaSetDevice(c->prm.device));
  double* d = nullptr;
  rpa_status st;
  if ((st = dev_alloc(c, (void**)&d, sizeof(double) * nw)) != RPA_OK) return st;
  CUDA_OK(c, cudaMemcpyAsync(d, omega, sizeof(double) * nw, cudaMemcpyHostToDevice, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  dev_free(c->omega_d);
  c->omega_d = d;
  c->nw_set = nw;
  return RPA_OK;
}

rpa_status rpa_energy_enqueue(rpa_ctx* c, int32_t nq, const int32_t* iqs) {
  if (!c) return RPA_ERR_ARG;
  if (nq < 1 || nq > kMaxIndex || !iqs) return fail(c, RPA_ERR_ARG, "bad rpa_energy_enqueue arguments");
  HOST_ARGS(c, iqs);
  if (!c->omega_d) return fail(c, RPA_ERR_STATE, "rpa_set_frequencies has not been called");
  CUDA_OK(c, cudaSetDevice(c->prm.device));
  ++c->stamp;
  for (int i = 0; i < nq; ++i) {
    rpa_status st = check_q_ready(c, iqs[i]);
    if (st != RPA_OK) return st;
  }
  choose_transform_grid(c, iqs, nq);
  return energy_enqueue(c, nq, iqs, c->nw_set, c->omega_d);
}

// ---- persistent batched launch of many instances (the graph's form)
// A unit is one (context, q-point) of the batch; a job is one k-block of a
// unit (rows [a0, a1) of transition t).  Consecutive jobs are packed into
// groups under an operand budget and the persistent kernel's job limit; per
// group: the pair densities and operand preparation of every job into a
// graph-owned pool, one persistent rank-k launch over all of the group's
// jobs, then the log-det of every unit whose last job was in the group.
struct BatchUnit {
  int ctx = 0, iq = 0, pos = 0;   // context index, q-point, position in its context's result arrays
  int job_begin = 0, job_end = 0; // jobs [begin, end)
  int g_first = 0, g_last = 0;    // groups of its first and last job
};
struct BatchJobPlan {
  int unit = 0, t = 0, a0 = 0, a1 = 0;
  int64_t P = 0;
  int NG = 0;
  size_t sb = 0;      // operand bytes
  size_t off = 0;     // offset in the pool
};

struct rpa_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t stream = nullptr;
  int device = 0;
  // persistent batched form
  bool persist = false;
  std::vector<BatchUnit> units;
  std::vector<BatchJobPlan> jobs;
  std::vector<std::pair<int, int>> groups;  // jobs [first, second)
  void* pool = nullptr;
  size_t pool_bytes = 0;
  int* dev = nullptr;          // [0] item counter, [1] error flag
  int** err_dst = nullptr;     // every context's error flag (device array)
  // batched log-dets: per group, the matrix descriptors (device copy, written
  // once before capture) and the host copy they were made from
  std::vector<LdMat*> ld_dev;
  std::vector<std::vector<LdMat>> ld_host;
};

namespace {

// Units, jobs and groups of a batch (host only; sizes from the contexts' state).
rpa_status plan_batch(rpa_graph* g, rpa_ctx* const* ctxs, int n, const int32_t* nq, const int32_t* iqs,
                      size_t budget) {
  g->units.clear();
  g->jobs.clear();
  g->groups.clear();
  g->pool_bytes = 0;
  int64_t off = 0;
  for (int i = 0; i < n; ++i) {
    rpa_ctx* c = ctxs[i];
    const int nw = c->nw_set;
    for (int u = 0; u < nq[i]; ++u) {
      const int iq = iqs[off + u];
      QPt& Q = c->qpts[iq];
      BatchUnit U;
      U.ctx = i;
      U.iq = iq;
      U.pos = u;
      U.job_begin = (int)g->jobs.size();
      for (size_t t = 0; t < Q.k_of.size(); ++t) {
        const int nL = (int)c->sets[Q.k_of[t]].L.size(), nR = (int)c->sets[Q.kq_of[t]].R.size();
        const int rows = rows_per_block(c, nL, nR, Q.NG, nw);
        for (int a0 = 0; a0 < nL; a0 += rows) {
          BatchJobPlan J;
          J.unit = (int)g->units.size();
          J.t = (int)t;
          J.a0 = a0;
          J.a1 = std::min(nL, a0 + rows);
          J.P = (int64_t)(J.a1 - a0) * nR;
          J.NG = Q.NG;
          if (J.P == 0) continue;
          J.sb = (herk_tc_scratch_bytes(J.P, J.NG, nw, 2, tc_fused(c) ? 1 : 0) + 255) / 256 * 256;
          g->jobs.push_back(J);
        }
      }
      U.job_end = (int)g->jobs.size();
      g->units.push_back(U);
    }
    off += nq[i];
  }
  // groups: consecutive jobs under the budget (a larger job forms its own group)
  const int maxj = herk_tc_batch_max_jobs();
  size_t used = 0;
  int first = 0;
  for (int j = 0; j < (int)g->jobs.size(); ++j) {
    BatchJobPlan& J = g->jobs[j];
    if (j > first && (used + J.sb > budget || j - first >= maxj)) {
      g->groups.push_back({first, j});
      first = j;
      used = 0;
    }
    J.off = used;
    used += J.sb;
    g->pool_bytes = std::max(g->pool_bytes, used);
  }
  if (!g->jobs.empty() || g->groups.empty()) g->groups.push_back({first, (int)g->jobs.size()});
  auto group_of = [&](int j) {
    for (int k = 0; k < (int)g->groups.size(); ++k)
      if (j < g->groups[k].second) return k;
    return (int)g->groups.size() - 1;
  };
  for (BatchUnit& U : g->units) {
    U.g_first = group_of(U.job_begin);
    U.g_last = U.job_end > U.job_begin ? group_of(U.job_end - 1) : U.g_first;
  }
  return RPA_OK;
}

// All device work of the batch on the shared stream (capturable).
rpa_status batched_enqueue(rpa_graph* g, rpa_ctx* const* ctxs, int n, const int32_t* nq, const int32_t* iqs) {
  rpa_status st;
  cudaStream_t s = ctxs[0]->stream;
  int64_t off = 0;
  for (int i = 0; i < n; ++i) {
    rpa_ctx* c = ctxs[i];
    ++c->stamp;
    choose_transform_grid(c, iqs + off, nq[i]);
    void *p_ld, *p_tr, *p_fl;
    if ((st = workspace(c, "res_ld", sizeof(double) * (size_t)nq[i] * c->nw_set, &p_ld)) != RPA_OK) return st;
    if ((st = workspace(c, "res_tr", sizeof(double) * (size_t)nq[i] * c->nw_set, &p_tr)) != RPA_OK) return st;
    if ((st = workspace(c, "res_flag", sizeof(int) * (size_t)nq[i], &p_fl)) != RPA_OK) return st;
    CUDA_OK(c, cudaMemsetAsync(c->dev_err, 0, sizeof(int), s));
    c->enq_iqs.assign(iqs + off, iqs + off + nq[i]);
    off += nq[i];
  }
  rpa_ctx* c0 = ctxs[0];
  CUDA_OK(c0, cudaMemsetAsync(g->dev + 1, 0, sizeof(int), s));
  // each context's log-det work buffer at its largest size up front, so its
  // address (held by the batched log-det descriptors) never changes
  {
    std::vector<int64_t> need(n, 0);
    for (const BatchUnit& U : g->units)
      need[U.ctx] = std::max(need[U.ctx], logdet_work_elems(ctxs[U.ctx]->nw_set, ctxs[U.ctx]->qpts[U.iq].NG));
    for (int i = 0; i < n; ++i) {
      void* p;
      if (need[i] && (st = workspace(ctxs[i], "chol", sizeof(double2) * (size_t)need[i], &p)) != RPA_OK) return st;
    }
  }
  std::vector<double2*> chi(g->units.size(), nullptr);
  for (int gi = 0; gi < (int)g->groups.size(); ++gi) {
    // units starting here: chi0 cleared, grids of their sets built
    for (size_t u = 0; u < g->units.size(); ++u) {
      const BatchUnit& U = g->units[u];
      if (U.g_first != gi) continue;
      rpa_ctx* c = ctxs[U.ctx];
      QPt& Q = c->qpts[U.iq];
      // a context's first q-point shares the chi0 buffer of its own evaluations
      const std::string key = U.pos == 0 ? std::string("chi") : "chiq" + std::to_string(U.iq);
      void* p;
      const size_t bytes = sizeof(double2) * (size_t)c->nw_set * Q.NG * Q.NG;
      if ((st = workspace(c, key.c_str(), bytes, &p)) != RPA_OK) return st;
      CUDA_OK(c, cudaMemsetAsync(p, 0, bytes, s));
      chi[u] = (double2*)p;
      for (size_t t = 0; t < Q.k_of.size(); ++t) {
        if ((st = build_grids(c, c->sets[Q.k_of[t]])) != RPA_OK) return st;
        if ((st = build_grids(c, c->sets[Q.kq_of[t]])) != RPA_OK) return st;
      }
    }
    // pair densities and operands of the group's jobs, then one persistent launch
    const int jb = g->groups[gi].first, je = g->groups[gi].second;
    std::vector<int64_t> P;
    std::vector<int> NG, nw;
    std::vector<void*> scr;
    std::vector<size_t> sb;
    std::vector<double2*> chis;
    std::vector<int> unit_of;
    int fused = -1;
    for (int j = jb; j < je; ++j) {
      const BatchJobPlan& J = g->jobs[j];
      const BatchUnit& U = g->units[J.unit];
      rpa_ctx* c = ctxs[U.ctx];
      QPt& Q = c->qpts[U.iq];
      Block<float> B;
      if ((st = pairs_block<float>(c, Q, J.t, J.a0, J.a1, c->omega_d, c->nw_set, B, 0)) != RPA_OK) return st;
      const int fz = tc_fused(c) ? 1 : 0;
      if (fused >= 0 && fz != fused) return fail(c, RPA_ERR_ARG, "the contexts of a batch differ in RPA_TUNE_TC_FUSE");
      fused = fz;
      void* p = (char*)g->pool + J.off;
      CUDA_OK(c, herk_tc_prepare((const float2*)B.N, B.P, B.NG, (const float*)B.w, c->nw_set, 2, fz, p, J.sb, s));
      P.push_back(J.P);
      NG.push_back(J.NG);
      nw.push_back(c->nw_set);
      scr.push_back(p);
      sb.push_back(J.sb);
      chis.push_back(chi[J.unit]);
      unit_of.push_back(J.unit);
    }
    if (!P.empty())
      CUDA_OK(c0, herk_tc_batch_run((int)P.size(), P.data(), NG.data(), nw.data(), scr.data(), sb.data(),
                                    unit_of.data(), chis.data(), fused, (int)c0->tune[RPA_TUNE_TC_FOLD],
                                    (int)c0->tune[RPA_TUNE_TC_FLUSH], c0->tune[RPA_TUNE_TC_WAIT_US], g->dev,
                                    g->dev + 1, s));
    // log-dets of the units that end here: the float-float ones of distinct
    // contexts as one batched factorisation, the others one by one
    std::vector<LdMat> mats;
    std::vector<int> in_batch;
    int maxNG = 0;
    for (size_t u = 0; u < g->units.size(); ++u) {
      const BatchUnit& U = g->units[u];
      if (U.g_last != gi) continue;
      rpa_ctx* c = ctxs[U.ctx];
      QPt& Q = c->qpts[U.iq];
      const int nw_ = c->nw_set;
      void* p_work;
      if ((st = workspace(c, "chol", sizeof(double2) * (size_t)logdet_work_elems(nw_, Q.NG), &p_work)) != RPA_OK)
        return st;
      double* ld = (double*)c->ws["res_ld"].p + (size_t)U.pos * nw_;
      double* tr = (double*)c->ws["res_tr"].p + (size_t)U.pos * nw_;
      int* fl = (int*)c->ws["res_flag"].p + U.pos;
      const bool shared = std::find(in_batch.begin(), in_batch.end(), U.ctx) != in_batch.end();
      if (ff_logdet(c) && !shared) {
        for (int w = 0; w < nw_; ++w) {
          LdMat m = logdet_mat((double2*)p_work, nw_, Q.NG, w);
          m.chi = chi[u] + (int64_t)w * Q.NG * Q.NG;
          m.v = Q.v_d;
          m.logdet = ld + w;
          m.trace = tr + w;
          m.flag = fl;
          mats.push_back(m);
        }
        in_batch.push_back(U.ctx);
        maxNG = std::max(maxNG, Q.NG);
        continue;
      }
      const LogdetStreams* la;
      if ((st = logdet_streams(c, &la)) != RPA_OK) return st;
      int64_t nl = 0;
      CUDA_OK(c, run_logdet(chi[u], Q.v_d, nw_, Q.NG, (double2*)p_work, ld, tr, fl, ff_logdet(c), s, &nl, la));
    }
    if (!mats.empty()) {
      if ((int)g->ld_dev.size() <= gi) {
        g->ld_dev.resize(g->groups.size(), nullptr);
        g->ld_host.resize(g->groups.size());
      }
      if (!g->ld_dev[gi]) {
        // first (uncaptured) pass: the descriptors go to the device once
        CUDA_OK(c0, cudaMalloc((void**)&g->ld_dev[gi], sizeof(LdMat) * mats.size()));
        CUDA_OK(c0, cudaMemcpy(g->ld_dev[gi], mats.data(), sizeof(LdMat) * mats.size(), cudaMemcpyHostToDevice));
        g->ld_host[gi] = mats;
      } else {
        const std::vector<LdMat>& h = g->ld_host[gi];
        bool same = h.size() == mats.size();
        for (size_t i = 0; same && i < h.size(); ++i)
          same = h[i].A == mats[i].A && h[i].Linv == mats[i].Linv && h[i].Linv_ff == mats[i].Linv_ff &&
                 h[i].Lp == mats[i].Lp && h[i].chi == mats[i].chi && h[i].v == mats[i].v &&
                 h[i].logdet == mats[i].logdet && h[i].trace == mats[i].trace && h[i].flag == mats[i].flag &&
                 h[i].NG == mats[i].NG;
        if (!same) return fail(c0, RPA_ERR_STATE, "batched log-det buffers moved between the warm-up and the capture");
      }
      int64_t nl = 0;
      CUDA_OK(c0, run_logdet_batch(g->ld_dev[gi], (int)mats.size(), maxNG, s, &nl));
    }
  }
  // a bounded wait that gave up reaches every context's flag
  CUDA_OK(c0, launch_or_flags(g->dev + 1, g->err_dst, n, s));
  return RPA_OK;
}
}  // namespace

rpa_status rpa_graph_create(rpa_ctx* const* ctxs, int32_t n, const int32_t* nq, const int32_t* iqs, rpa_graph** out) {
  if (!ctxs || n < 1 || !nq || !iqs || !out) return RPA_ERR_ARG;
  if (!host_readable(ctxs) || !ctxs[0]) return RPA_ERR_ARG;
  if (!on_device(ctxs[0]->prm.device)) return RPA_ERR_CUDA;
  if (!host_readable(nq) || !host_readable(iqs) || !host_readable(out)) return RPA_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || nq[i] < 1) return RPA_ERR_ARG;
    if (ctxs[i]->stream != ctxs[0]->stream || ctxs[i]->prm.device != ctxs[0]->prm.device)
      return fail(ctxs[i], RPA_ERR_ARG, "all contexts of a graph must share one stream and device");
    if (!ctxs[0]->prm.stream) return fail(ctxs[i], RPA_ERR_ARG, "a graph needs a caller-provided stream");
    if (!ctxs[i]->omega_d) return fail(ctxs[i], RPA_ERR_STATE, "rpa_set_frequencies has not been called");
  }
  cudaStream_t s = ctxs[0]->stream;
  if (cudaSetDevice(ctxs[0]->prm.device) != cudaSuccess) return RPA_ERR_CUDA;
  int64_t off = 0;
  for (int i = 0; i < n; ++i) {
    for (int u = 0; u < nq[i]; ++u)
      if (rpa_status st = check_q_ready(ctxs[i], iqs[off + u]); st != RPA_OK) return st;
    off += nq[i];
  }
  // the persistent form: every context in the two-term split mode, not switched off
  bool persist = ctxs[0]->tune[RPA_TUNE_BATCH_PERSIST] == 1;
  for (int i = 0; i < n; ++i)
    persist = persist && ctxs[i]->prm.precision == RPA_BF16X2 && ctxs[i]->tune[RPA_TUNE_TC_PIPE] == 0 &&
              ctxs[i]->tune[RPA_TUNE_TC_FUSE] == ctxs[0]->tune[RPA_TUNE_TC_FUSE];
  rpa_graph* g = new rpa_graph();
  g->stream = s;
  g->device = ctxs[0]->prm.device;
  g->persist = persist;
  auto bail = [&](rpa_status st) {
    cudaGetLastError();
    rpa_graph_destroy(g);
    return st;
  };
  if (persist) {
    std::vector<int*> dst(n);
    for (int i = 0; i < n; ++i) dst[i] = ctxs[i]->dev_err;
    if (cudaMalloc(&g->dev, 2 * sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&g->err_dst, sizeof(int*) * n) != cudaSuccess)
      return bail(fail(ctxs[0], RPA_ERR_OOM, "batched graph buffers could not be allocated"));
    // the operand budget is an upper bound: where the device has less free,
    // halve it (more, smaller groups) down to the largest single job
    size_t budget = (size_t)ctxs[0]->tune[RPA_TUNE_BATCH_MB] << 20;
    for (;;) {
      plan_batch(g, ctxs, n, nq, iqs, budget);
      if (!g->pool_bytes || cudaMalloc(&g->pool, g->pool_bytes) == cudaSuccess) break;
      cudaGetLastError();
      g->pool = nullptr;
      size_t largest = 0;
      for (const BatchJobPlan& J : g->jobs) largest = std::max(largest, J.sb);
      if (budget <= largest)
        return bail(fail(ctxs[0], RPA_ERR_OOM, "batched graph operand pool (%zu bytes) could not be allocated",
                         g->pool_bytes));
      budget = std::max(budget / 2, largest);
    }
    if (cudaMemcpy(g->err_dst, dst.data(), sizeof(int*) * n, cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(RPA_ERR_CUDA);
  }
  // warm-up outside the capture: sizes every workspace and device table
  off = 0;
  if (persist) {
    if (rpa_status st = batched_enqueue(g, ctxs, n, nq, iqs); st != RPA_OK) return bail(st);
  } else {
    for (int i = 0; i < n; ++i) {
      rpa_status st = rpa_energy_enqueue(ctxs[i], nq[i], iqs + off);
      if (st != RPA_OK) return bail(st);
      off += nq[i];
    }
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return bail(fail(ctxs[0], RPA_ERR_CUDA, "warm-up run failed"));
  std::vector<bool> prof(n);
  for (int i = 0; i < n; ++i) {
    prof[i] = ctxs[i]->profiling;
    ctxs[i]->profiling = false;
  }
  rpa_status st = RPA_OK;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    st = fail(ctxs[0], RPA_ERR_CUDA, "cudaStreamBeginCapture failed");
  } else {
    off = 0;
    if (persist) {
      st = batched_enqueue(g, ctxs, n, nq, iqs);
    } else {
      for (int i = 0; i < n && st == RPA_OK; ++i) {
        st = rpa_energy_enqueue(ctxs[i], nq[i], iqs + off);
        off += nq[i];
      }
    }
    const cudaError_t e = cudaStreamEndCapture(s, &g->graph);
    if (st == RPA_OK && e != cudaSuccess) st = fail(ctxs[0], RPA_ERR_CUDA, "capture failed: %s", cudaGetErrorString(e));
    if (st == RPA_OK && cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess)
      st = fail(ctxs[0], RPA_ERR_CUDA, "cudaGraphInstantiate failed");
  }
  for (int i = 0; i < n; ++i) ctxs[i]->profiling = prof[i];
  if (st != RPA_OK) {
    cudaGetLastError();
    rpa_graph_destroy(g);
    return st;
  }
  *out = g;
  return RPA_OK;
}

rpa_status rpa_graph_launch(rpa_graph* g) {
  if (!g || !g->exec) return RPA_ERR_ARG;
  if (cudaSetDevice(g->device) != cudaSuccess) return RPA_ERR_CUDA;
  return cudaGraphLaunch(g->exec, g->stream) == cudaSuccess ? RPA_OK : RPA_ERR_CUDA;
}

void rpa_graph_destroy(rpa_graph* g) {
  if (!g) return;
  cudaSetDevice(g->device);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->pool) cudaFree(g->pool);
  for (LdMat* p : g->ld_dev)
    if (p) cudaFree(p);
  if (g->dev) cudaFree(g->dev);
  if (g->err_dst) cudaFree(g->err_dst);
  delete g;
}

rpa_status rpa_energy_collect(rpa_ctx* c, const double* wq, const double* W, double* Ec, double* terms) {
  if (!c) return RPA_ERR_ARG;
  if (!wq || !W || !Ec) return fail(c, RPA_ERR_ARG, "bad rpa_energy_collect arguments");
  HOST_ARGS(c, wq, W, Ec, terms);
  CUDA_OK(c, cudaSetDevice(c->prm.device));
  return energy_collect(c, c->nw_set, wq, W, Ec, terms);
}

rpa_status rpa_energy_backward(rpa_ctx* c, int32_t nq, const int32_t* iqs, const double* wq, int32_t nw,
                               const double* omega, const double* W, double dEc, double* Ec, int32_t nsets,
                               const int32_t* set_ids, double* const* dC, double* const* dP, double* const* dchi) {
  if (!c) return RPA_ERR_ARG;
  if (nq < 1 || nq > kMaxIndex || !iqs || !wq || nw < 1 || nw > 4096 || !omega || !W || nsets < 0 ||
      (nsets > 0 && !set_ids) || !std::isfinite(dEc))
    return fail(c, RPA_ERR_ARG, "bad rpa_energy_backward arguments");
  HOST_ARGS(c, iqs, wq, omega, W, Ec, set_ids, dC, dP, dchi);
  CUDA_OK(c, cudaSetDevice(c->prm.device));
  prof_begin(c);
  ++c->stamp;
  for (int i = 0; i < nq; ++i) {
    rpa_status st = check_q_ready(c, iqs[i]);
    if (st != RPA_OK) return st;
  }
  choose_transform_grid(c, iqs, nq);
  rpa_status st;
  if (c->prm.precision == RPA_FP64)
    st = energy_backward_T<double>(c, nq, iqs, wq, nw, omega, W, dEc, Ec, nsets, set_ids, dC, dP, dchi);
  else
    st = energy_backward_T<float>(c, nq, iqs, wq, nw, omega, W, dEc, Ec, nsets, set_ids, dC, dP, dchi);
  if (st != RPA_OK) return st;
  prof_end(c);
  return RPA_OK;
}

rpa_status rpa_set_profiling(rpa_ctx* c, int32_t enable) {
  if (!c) return RPA_ERR_ARG;
  c->profiling = enable != 0;
  return RPA_OK;
}

rpa_status rpa_set_tuning(rpa_ctx* c, int32_t param, int64_t value) {
  if (!c) return RPA_ERR_ARG;
  switch (param) {
    case RPA_TUNE_TC_FOLD:
    case RPA_TUNE_TC_FLUSH:
      if (value < 1 || value > (1 << 20)) return fail(c, RPA_ERR_ARG, "fold interval %lld out of range", (long long)value);
      break;
    case RPA_TUNE_PAIR_CHUNK:
      if (value < 0 || value > (1ll << 30)) return fail(c, RPA_ERR_ARG, "pair chunk %lld out of range", (long long)value);
      break;
    case RPA_TUNE_PD_GRID:
      if (value != 0 && value != 1) return fail(c, RPA_ERR_ARG, "transform grid choice must be 0 or 1");
      break;
    case RPA_TUNE_TC_PIPE:
      if (value != 0 && value != 1) return fail(c, RPA_ERR_ARG, "tensor-core pipeline shape must be 0 or 1");
      break;
    case RPA_TUNE_LOGDET:
      if (value < 0 || value > 2) return fail(c, RPA_ERR_ARG, "log-det update choice must be 0, 1 or 2");
      break;
    case RPA_TUNE_PAW_TC:
      if (value != 0 && value != 1) return fail(c, RPA_ERR_ARG, "PAW product choice must be 0 or 1");
      break;
    case RPA_TUNE_TC_FUSE:
      if (value != 0 && value != 1) return fail(c, RPA_ERR_ARG, "fused weighting choice must be 0 or 1");
      break;
    case RPA_TUNE_PD_FUSE:
      if (value != 0 && value != 1) return fail(c, RPA_ERR_ARG, "fused pair-density stage choice must be 0 or 1");
      break;
    case RPA_TUNE_BATCH_PERSIST:
      if (value != 0 && value != 1) return fail(c, RPA_ERR_ARG, "batched launch choice must be 0 or 1");
      break;
    case RPA_TUNE_GAMMA:
      if (value < 0 || value > 2) return fail(c, RPA_ERR_ARG, "gradient precision choice must be 0, 1 or 2");
      break;
    case RPA_TUNE_TC_PAIR:
      if (value < 0 || value > 2) return fail(c, RPA_ERR_ARG, "paired rank-k launch must be 0, 1 or 2");
      break;
    case RPA_TUNE_PD_FACT:
      if (value != 0 && value != 1) return fail(c, RPA_ERR_ARG, "factorised pair-density axes must be 0 or 1");
      break;
    case RPA_TUNE_LD_OVERLAP:
      if (value != 0 && value != 1) return fail(c, RPA_ERR_ARG, "log-det overlap must be 0 or 1");
      break;
    case RPA_TUNE_BATCH_MB:
      if (value < 1 || value > (1 << 22)) return fail(c, RPA_ERR_ARG, "batch group budget %lld MiB out of range", (long long)value);
      break;
    case RPA_TUNE_TC_WAIT_US:
      if (value < 1000 || value > 60000000)
        return fail(c, RPA_ERR_ARG, "wait limit %lld us out of range", (long long)value);
      break;
    case RPA_TUNE_TC_STALL:
      if (value < 0 || value > (1 << 30)) return fail(c, RPA_ERR_ARG, "stall stage %lld out of range", (long long)value);
      break;
    case RPA_TUNE_OPERAND_MB:
      if (value < 16 || value > (1 << 20)) return fail(c, RPA_ERR_ARG, "operand budget %lld MB out of range", (long long)value);
      break;
    default:
      return fail(c, RPA_ERR_ARG, "unknown tuning parameter %d", param);
  }
  c->tune[param] = value;
  return RPA_OK;
}

rpa_status rpa_get_profile(const rpa_ctx* c, double* ms, int64_t* launches) {
  if (!c) return RPA_ERR_ARG;
  if (!on_device(c->prm.device)) return RPA_ERR_CUDA;
  if (!host_readable(ms) || !host_readable(launches)) return RPA_ERR_ARG;
  for (int i = 0; i < RPA_NSTAGES; ++i) {
    if (ms) ms[i] = c->prof_ms[i];
    if (launches) launches[i] = c->prof_launch[i];
  }
  return RPA_OK;
}

}  // extern "C"
