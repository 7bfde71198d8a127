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
#include "rpa.h"
#include "rpa_internal.h"

namespace rpa {

constexpr int CB = 32;  // panel width
constexpr int UT = 64;  // update tile edge

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
    A[id] = a;
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

__global__ void __launch_bounds__(256) chol_diag_kernel(double2* __restrict__ A, int NG, int k0, int b,
                                                        double* __restrict__ logdet, int* __restrict__ flag) {
  __shared__ double2 L[CB][CB + 1];
  __shared__ double ld;
  const int w = blockIdx.x;
  double2* Aw = A + (int64_t)w * NG * NG;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e % b;
    if (j <= i) L[i][j] = Aw[(int64_t)(k0 + i) * NG + k0 + j];
  }
  if (threadIdx.x == 0) ld = 0.0;
  __syncthreads();
  for (int c = 0; c < b; ++c) {
    if (threadIdx.x == 0) {
      double piv = L[c][c].x;
      if (!(piv > 0.0)) {
        atomicExch(flag, 1);
        piv = 1.0;
      }
      ld += log(piv);
      L[c][c] = make_double2(sqrt(piv), 0.0);
    }
    __syncthreads();
    const double dinv = 1.0 / L[c][c].x;
    for (int i = c + 1 + threadIdx.x; i < b; i += blockDim.x) {
      L[i][c].x *= dinv;
      L[i][c].y *= dinv;
    }
    __syncthreads();
    const int m = b - c - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = c + 1 + e / m, j = c + 1 + e % m;
      if (j <= i) {
        const double2 x = L[i][c], y = L[j][c];
        // L_ij -= x * conj(y)
        L[i][j].x -= x.x * y.x + x.y * y.y;
        L[i][j].y -= x.y * y.x - x.x * y.y;
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e % b;
    if (j <= i) Aw[(int64_t)(k0 + i) * NG + k0 + j] = L[i][j];
  }
  if (threadIdx.x == 0) logdet[w] += ld;
}

constexpr int TR = 32;  // rows per triangular-solve CTA

__global__ void __launch_bounds__(TR) chol_trsm_kernel(double2* __restrict__ A, int NG, int k0, int b) {
  __shared__ double2 Lk[CB][CB + 1];
  __shared__ double2 X[TR][CB + 1];
  const int w = blockIdx.y;
  double2* Aw = A + (int64_t)w * NG * NG;
  const int i0 = k0 + b + blockIdx.x * TR;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e % b;
    Lk[i][j] = (j <= i) ? Aw[(int64_t)(k0 + i) * NG + k0 + j] : make_double2(0.0, 0.0);
  }
  for (int e = threadIdx.x; e < TR * b; e += blockDim.x) {
    const int r = e / b, j = e % b;
    X[r][j] = (i0 + r < NG) ? Aw[(int64_t)(i0 + r) * NG + k0 + j] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int r = threadIdx.x;
  if (i0 + r < NG) {
    // solve x L^H = a: x_j = (a_j - sum_{l<j} x_l conj(L_jl)) / L_jj
    for (int j = 0; j < b; ++j) {
      double2 s = X[r][j];
      for (int l = 0; l < j; ++l) {
        const double2 x = X[r][l], y = Lk[j][l];
        s.x -= x.x * y.x + x.y * y.y;
        s.y -= x.y * y.x - x.x * y.y;
      }
      const double dinv = 1.0 / Lk[j][j].x;
      X[r][j] = make_double2(s.x * dinv, s.y * dinv);
    }
    for (int j = 0; j < b; ++j) Aw[(int64_t)(i0 + r) * NG + k0 + j] = X[r][j];
  }
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

__global__ void add_terms_kernel(const double* __restrict__ ld, const double* __restrict__ tr, int nw,
                                 double* __restrict__ terms) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w < nw) terms[w] = ld[w] + tr[w];
}

static inline int gridc(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b > 152 * 64 ? 152 * 64 : (b < 1 ? 1 : b));
}

cudaError_t run_logdet(const double2* chi, const double* v, int nw, int NG, double2* work, double* logdet,
                       double* trace, int* flag, cudaStream_t s, int64_t* launches) {
  cudaError_t e;
  int64_t nl = 0;
  const int upd_smem = 2 * CB * UT * (int)sizeof(double2);
  if ((e = cudaFuncSetAttribute(chol_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, upd_smem)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(logdet, 0, sizeof(double) * nw, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(flag, 0, sizeof(int), s)) != cudaSuccess) return e;
  const int64_t total = (int64_t)nw * NG * NG;
  chol_form_kernel<<<gridc(total), 256, 0, s>>>(chi, v, nw, NG, work);
  trace_kernel<<<nw, 256, 0, s>>>(chi, v, NG, trace);
  nl += 2;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int k0 = 0; k0 < NG; k0 += CB) {
    const int b = (NG - k0) < CB ? (NG - k0) : CB;
    chol_diag_kernel<<<nw, 256, 0, s>>>(work, NG, k0, b, logdet, flag);
    ++nl;
    const int rest = NG - k0 - b;
    if (rest > 0) {
      chol_trsm_kernel<<<dim3((rest + TR - 1) / TR, nw), TR, 0, s>>>(work, NG, k0, b);
      const int nt = (rest + UT - 1) / UT;
      chol_update_kernel<<<dim3(nt * (nt + 1) / 2, nw), 256, upd_smem, s>>>(work, NG, k0, b);
      nl += 2;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (launches) *launches += nl;
  return cudaSuccess;
}

// ---------------------------------------------------------------- allocation-free entry point
// Scratch of rpa_logdet_noalloc: the Cholesky work matrix (up to
// kNoAllocMaxElems complex elements) followed by the per-frequency log-det and
// trace accumulators and the pivot flag.  It lives for the life of the process
// on every device that loads the library (16 MiB + 2 KiB).
constexpr int64_t kNoAllocMaxElems = (int64_t)1 << 20;
constexpr int kNoAllocMaxNw = 64;
constexpr int64_t kNoAllocSlots = kNoAllocMaxElems + kNoAllocMaxNw + 1;  // double2 slots
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
  double* ld = (double*)(work + kNoAllocMaxElems);
  double* tr = ld + kNoAllocMaxNw;
  int* flag = (int*)(tr + kNoAllocMaxNw);
  // run_logdet clears the log-det accumulators and the flag itself; the work
  // matrix is fully rewritten from chi before it is read
  if (run_logdet((const double2*)chi, v, nw, ng, work, ld, tr, flag, s, nullptr) != cudaSuccess) return RPA_ERR_CUDA;
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
