// Plane-wave <-> real-space transforms of the RPA hot path, without cuFFT.
//
//  * Wavefunctions to the grid (Eq. 8; Table 1 step 3): the coefficients are
//    scattered into their Miller box and transformed axis by axis with pruned
//    DFTs (only the occupied Miller range is summed).
//  * Pair densities (Eq. 10; Table 1 steps 5-6): the product
//    conj(u_nk(r)) u_m,k+q(r) is fused into the first (slowest-axis) DFT, the
//    middle axis follows, and the fastest axis is evaluated only on the
//    response sphere g = G + G0 (the "mapG" gather of step 6 fused into the
//    transform).  The PAW term of Eq. 6 (steps 8-9) is then added by one
//    complex GEMM per occupied band (paw_gemm_kernel) from the factorised form
//    sum_(a,j) P_mj R^a_n(j,G) with R^a_n(j,G) = sum_i conj(P_ni) Q^a_ij(G)
//    (paw_R_kernel), which equals the paper's outer-product-then-contract
//    order in exact arithmetic.
//
// Twiddles come from a table tw[t] = exp(2 pi i t / N), t in [0, N), filled
// with sincospi in double precision; every phase index is reduced exactly in
// integer arithmetic, so no angle is ever rounded before the table lookup.
#include "rpa_internal.h"

#include <algorithm>

namespace rpa {

static inline int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 64) b = 152 * 64;
  if (b < 1) b = 1;
  return (int)b;
}

__host__ __device__ inline int pmod(int64_t a, int n) {
  int64_t r = a % n;
  return (int)(r < 0 ? r + n : r);
}

template <typename T>
__device__ inline void fill_twiddles(c2<T>* tw, int N) {
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)t / (double)N, &s, &c);
    tw[t] = mk<T>((T)c, (T)s);
  }
  __syncthreads();
}

// tw[t] = exp(2 pi i t / N), t < N: the values fill_twiddles forms, once in
// global memory for kernels with many short blocks
template <typename T>
__global__ void twiddle_line_kernel(c2<T>* __restrict__ tw, int N) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N; t += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)t / (double)N, &s, &c);
    tw[t] = mk<T>((T)c, (T)s);
  }
}

template <typename T>
cudaError_t launch_twiddle_line(c2<T>* tw, int N, cudaStream_t s) {
  twiddle_line_kernel<T><<<(N + 255) / 256, 256, 0, s>>>(tw, N);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- generic axis DFT
template <typename T, int TO>
__global__ void __launch_bounds__(256) dft_axis_kernel(const c2<T>* __restrict__ in, c2<T>* __restrict__ out,
                                                       int64_t rows, int Lin, int Lout, int B, int N,
                                                       int in_off, int out_off, int sign) {
  extern __shared__ unsigned char smem_raw[];
  c2<T>* tw = reinterpret_cast<c2<T>*>(smem_raw);
  fill_twiddles<T>(tw, N);
  const int nchunk = (Lout + TO - 1) / TO;
  const int64_t total = rows * nchunk * (int64_t)B;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(id % B);
    int64_t r = id / B;
    const int oc = (int)(r % nchunk);
    r /= nchunk;
    const int o0 = oc * TO;
    int idx[TO], step[TO];
    c2<T> acc[TO];
#pragma unroll
    for (int t = 0; t < TO; ++t) {
      const int64_t j = out_off + o0 + t;
      step[t] = pmod(sign * j, N);
      idx[t] = pmod(sign * (int64_t)in_off * j, N);
      acc[t] = mk<T>(0, 0);
    }
    const c2<T>* src = in + (r * Lin) * B + c;
    for (int i = 0; i < Lin; ++i) {
      const c2<T> x = src[(int64_t)i * B];
#pragma unroll
      for (int t = 0; t < TO; ++t) {
        cmac<T>(acc[t], x, tw[idx[t]]);
        idx[t] += step[t];
        if (idx[t] >= N) idx[t] -= N;
      }
    }
    c2<T>* dst = out + (r * Lout + o0) * B + c;
#pragma unroll
    for (int t = 0; t < TO; ++t)
      if (o0 + t < Lout) dst[(int64_t)t * B] = acc[t];
  }
}

template <typename T>
cudaError_t launch_dft_axis(const c2<T>* in, c2<T>* out, int64_t batch, int A, int Lin, int Lout,
                            int B, int N, int in_off, int out_off, int sign, cudaStream_t s) {
  constexpr int TO = 4;  // outputs a thread (8 measured slower)
  const int64_t rows = batch * A;
  const int64_t total = rows * ((Lout + TO - 1) / TO) * (int64_t)B;
  if (total == 0) return cudaSuccess;
  dft_axis_kernel<T, TO><<<grid_for(total, 256), 256, N * sizeof(c2<T>), s>>>(in, out, rows, Lin, Lout, B, N,
                                                                            in_off, out_off, sign);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- scatter into Miller box
template <typename T>
__global__ void scatter_box_kernel(const double2* __restrict__ C, int nb, int npw, const int* __restrict__ pos,
                                   int64_t box, c2<T>* __restrict__ out) {
  const int64_t total = (int64_t)nb * npw;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(id / npw);
    const int q = (int)(id % npw);
    const double2 v = C[id];
    out[(int64_t)b * box + pos[q]] = mk<T>((T)v.x, (T)v.y);
  }
}

template <typename T>
cudaError_t launch_scatter_box(const double2* C, int nb, int npw, const int* pos, int64_t box, c2<T>* out,
                               cudaStream_t s) {
  const int64_t total = (int64_t)nb * npw;
  if (total == 0) return cudaSuccess;
  scatter_box_kernel<T><<<grid_for(total, 256), 256, 0, s>>>(C, nb, npw, pos, box, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- pair density stage A
// T1[pl][o][j23] = sum_j1 conj(u_n(j1, j23)) u_m(j1, j23) exp(-2 pi i g1 j1 / N1), g1 = g1lo + o
// The twiddle matrices tw[oc][j][o] = exp(-2 pi i (lo + 16 oc + o) j / N) of the
// pruned outputs are built once per transform (FP64 sincospi of an exactly
// reduced integer phase) in global memory; each block copies its chunk into
// shared memory, where every thread of a warp reads the same entry (broadcast).
template <typename T>
__global__ void twiddle_matrix_kernel(c2<T>* __restrict__ tw, int N, int lo, int n, int NO, int nchunk) {
  const int64_t total = (int64_t)nchunk * N * NO;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int oc = (int)(e / ((int64_t)N * NO));
    const int r = (int)(e % ((int64_t)N * NO));
    const int j = r / NO, o = oc * NO + r % NO;
    if (o < n) {
      const int t = pmod(-(int64_t)(lo + o) * j, N);
      double s, c;
      sincospi(2.0 * (double)t / (double)N, &s, &c);
      tw[e] = mk<T>((T)c, (T)s);
    } else {
      tw[e] = mk<T>(0, 0);
    }
  }
}

template <typename T>
cudaError_t launch_twiddle_matrix(c2<T>* tw, int N, int lo, int n, cudaStream_t s) {
  constexpr int NO = 16;
  const int nchunk = (n + NO - 1) / NO;
  const int64_t total = (int64_t)nchunk * N * NO;
  if (total == 0) return cudaSuccess;
  twiddle_matrix_kernel<T><<<grid_for(total, 256), 256, 0, s>>>(tw, N, lo, n, NO, nchunk);
  return cudaGetLastError();
}

template <typename T>
__device__ inline void load_twiddle_matrix(c2<T>* tw, const c2<T>* __restrict__ src, int count) {
  for (int e = threadIdx.x; e < count; e += blockDim.x) tw[e] = src[e];
  __syncthreads();
}

// Each thread owns one (j2, j3) line point and PP consecutive pairs, and keeps
// all NO outputs g1 of each pair in registers while it streams j1.
// Twiddle tables are stored with a row stride of TS = 16 outputs; a kernel
// instance computes NO <= 16 outputs per chunk (NO = 16 for several chunks).
constexpr int TS = 16;

// Per-thread cp.async ring: the transform kernels stream one grid line per
// thread, so each thread prefetches its own next PF-1 slices into private
// shared-memory slots (no block barrier needed) and the loads of several
// iterations are in flight at once.
template <typename T>
__device__ __forceinline__ void cp_async_elem(c2<T>* dst_smem, const c2<T>* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst_smem);
  if constexpr (sizeof(c2<T>) == 16)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// byte offset of the ring after a twiddle table of n entries
template <typename T>
__host__ __device__ constexpr int ring_offset(int n) {
  return (int)(((size_t)n * TS * sizeof(c2<T>) + 15) / 16 * 16);
}
constexpr int RING_PF = 4;       // stages of the ring

// Pair of chunk slot pl: a chunk holds nrow consecutive occupied rows of the
// block and np / nrow consecutive unoccupied bands from p0 (row 0), rows
// fastest, so neighbouring threads share an unoccupied band's grid; nrow = 1
// is the contiguous range p0 + pl.
__host__ __device__ inline int64_t chunk_pair(int pl, int64_t p0, int nrow, int nR) {
  return (int64_t)(pl % nrow) * nR + p0 + pl / nrow;
}
constexpr int RING_THREADS = 256;

template <typename T, int NO, int PP, int PF>
__global__ void __launch_bounds__(256) pd_stageA_kernel(const c2<T>* __restrict__ Uk, const c2<T>* __restrict__ Ukp,
                                                        int64_t Nr, int N1, int N23, const int* __restrict__ Lidx,
                                                        const int* __restrict__ Ridx, int nR, int64_t p0, int np,
                                                        int nrow, const c2<T>* __restrict__ twg, int n1,
                                                        c2<T>* __restrict__ T1) {
  extern __shared__ unsigned char smem_raw[];
  c2<T>* tw = reinterpret_cast<c2<T>*>(smem_raw);
  const int nchunk = (n1 + TS - 1) / TS;
  const int ngrp = (np + PP - 1) / PP;
  for (int oc = 0; oc < nchunk; ++oc) {
    const int o0 = oc * TS;
    const int nout = min(NO, n1 - o0);
    if (oc) __syncthreads();
    load_twiddle_matrix<T>(tw, twg + (int64_t)oc * N1 * TS, N1 * TS);
    const int64_t total = (int64_t)ngrp * N23;
    for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
      const int j23 = (int)(id % N23);
      const int grp = (int)(id / N23);
      const c2<T>* un[PP];
      const c2<T>* um[PP];
#pragma unroll
      for (int q = 0; q < PP; ++q) {
        const int pl = min(grp * PP + q, np - 1);
        const int64_t p = chunk_pair(pl, p0, nrow, nR);
        un[q] = Uk + (int64_t)Lidx[p / nR] * Nr + j23;
        um[q] = Ukp + (int64_t)Ridx[p % nR] * Nr + j23;
      }
      c2<T> acc[PP][NO];
#pragma unroll
      for (int q = 0; q < PP; ++q)
#pragma unroll
        for (int t = 0; t < NO; ++t) acc[q][t] = mk<T>(0, 0);
      if constexpr (PF > 1) {
        // slot (stage st, value v) of this thread: ring[(st * 2 PP + v) * 256 + tid]
        c2<T>* my = reinterpret_cast<c2<T>*>(smem_raw + ring_offset<T>(N1)) + threadIdx.x;
        auto issue = [&](int j) {
          const int st = j % PF;
#pragma unroll
          for (int q = 0; q < PP; ++q) {
            cp_async_elem<T>(my + (st * 2 * PP + 2 * q) * RING_THREADS, un[q] + (int64_t)j * N23);
            cp_async_elem<T>(my + (st * 2 * PP + 2 * q + 1) * RING_THREADS, um[q] + (int64_t)j * N23);
          }
        };
#pragma unroll
        for (int j = 0; j < PF - 1; ++j) {
          if (j < N1) issue(j);
          cp_async_commit();
        }
        for (int j1 = 0; j1 < N1; ++j1) {
          if (j1 + PF - 1 < N1) issue(j1 + PF - 1);
          cp_async_commit();
          cp_async_wait<PF - 1>();  // the group of slice j1 has landed
          const int st = j1 % PF;
          c2<T> x[PP];
#pragma unroll
          for (int q = 0; q < PP; ++q)
            x[q] = cj_mul<T>(my[(st * 2 * PP + 2 * q) * RING_THREADS], my[(st * 2 * PP + 2 * q + 1) * RING_THREADS]);
          const c2<T>* twj = tw + j1 * TS;
#pragma unroll
          for (int t = 0; t < NO; ++t) {
            const c2<T> f = twj[t];
#pragma unroll
            for (int q = 0; q < PP; ++q) cmac<T>(acc[q][t], x[q], f);
          }
        }
      } else {
        // the next j1 slice of both grids is loaded while the current one is used
        c2<T> nxt_n[PP], nxt_m[PP];
#pragma unroll
        for (int q = 0; q < PP; ++q) {
          nxt_n[q] = un[q][0];
          nxt_m[q] = um[q][0];
        }
        for (int j1 = 0; j1 < N1; ++j1) {
          c2<T> x[PP];
#pragma unroll
          for (int q = 0; q < PP; ++q) x[q] = cj_mul<T>(nxt_n[q], nxt_m[q]);
          if (j1 + 1 < N1) {
#pragma unroll
            for (int q = 0; q < PP; ++q) {
              nxt_n[q] = un[q][(int64_t)(j1 + 1) * N23];
              nxt_m[q] = um[q][(int64_t)(j1 + 1) * N23];
            }
          }
          const c2<T>* twj = tw + j1 * TS;
#pragma unroll
          for (int t = 0; t < NO; ++t) {
            const c2<T> f = twj[t];
#pragma unroll
            for (int q = 0; q < PP; ++q) cmac<T>(acc[q][t], x[q], f);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < PP; ++q) {
        const int pl = grp * PP + q;
        if (pl < np) {
          c2<T>* dst = T1 + ((int64_t)pl * n1 + o0) * N23 + j23;
#pragma unroll
          for (int t = 0; t < NO; ++t)
            if (t < nout) dst[(int64_t)t * N23] = acc[q][t];
        }
      }
    }
  }
}

template <typename T, int NO, int PF>
static cudaError_t launch_stageA_pf(const c2<T>* Uk, const c2<T>* Ukp, int64_t Nr, int N1, int N23, const int* Lidx,
                                    const int* Ridx, int nR, int64_t p0, int np, int nrow, const c2<T>* tw, int n1,
                                    c2<T>* T1, cudaStream_t s) {
  constexpr int PP = sizeof(T) == 4 ? 2 : 1;
  const int64_t total = (int64_t)((np + PP - 1) / PP) * N23;
  if (total == 0) return cudaSuccess;
  const int smem = PF > 1 ? ring_offset<T>(N1) + PF * 2 * PP * RING_THREADS * (int)sizeof(c2<T>)
                          : N1 * TS * (int)sizeof(c2<T>);
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(pd_stageA_kernel<T, NO, PP, PF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  pd_stageA_kernel<T, NO, PP, PF><<<grid_for(total, 256), 256, smem, s>>>(Uk, Ukp, Nr, N1, N23, Lidx, Ridx, nR, p0,
                                                                         np, nrow, tw, n1, T1);
  return cudaGetLastError();
}

// the ring needs PF * 2 PP * 256 slots next to the twiddle table; very long
// axes (table beyond 160 KB) fall back to one-slice register prefetch
template <typename T, int NO>
static cudaError_t launch_stageA_no(const c2<T>* Uk, const c2<T>* Ukp, int64_t Nr, int N1, int N23, const int* Lidx,
                                    const int* Ridx, int nR, int64_t p0, int np, int nrow, const c2<T>* tw, int n1,
                                    c2<T>* T1, cudaStream_t s) {
  if (ring_offset<T>(N1) <= 160 * 1024)
    return launch_stageA_pf<T, NO, RING_PF>(Uk, Ukp, Nr, N1, N23, Lidx, Ridx, nR, p0, np, nrow, tw, n1, T1, s);
  return launch_stageA_pf<T, NO, 1>(Uk, Ukp, Nr, N1, N23, Lidx, Ridx, nR, p0, np, nrow, tw, n1, T1, s);
}

// compute width: the smallest of 8, 12, 14, 16 that holds all outputs (16 with chunks beyond)
static inline int width_for(int n) { return n <= 8 ? 8 : n <= 12 ? 12 : n <= 14 ? 14 : 16; }

template <typename T>
cudaError_t launch_pd_stageA(const c2<T>* Uk, const c2<T>* Ukp, int64_t Nr, int N1, int N23, const int* Lidx,
                             const int* Ridx, int nR, int64_t p0, int np, int nrow, const c2<T>* tw, int n1, c2<T>* T1,
                             cudaStream_t s) {
  if (nrow < 1 || np % nrow) return cudaErrorInvalidValue;
  switch (width_for(n1)) {
    case 8: return launch_stageA_no<T, 8>(Uk, Ukp, Nr, N1, N23, Lidx, Ridx, nR, p0, np, nrow, tw, n1, T1, s);
    case 12: return launch_stageA_no<T, 12>(Uk, Ukp, Nr, N1, N23, Lidx, Ridx, nR, p0, np, nrow, tw, n1, T1, s);
    case 14: return launch_stageA_no<T, 14>(Uk, Ukp, Nr, N1, N23, Lidx, Ridx, nR, p0, np, nrow, tw, n1, T1, s);
    default: return launch_stageA_no<T, 16>(Uk, Ukp, Nr, N1, N23, Lidx, Ridx, nR, p0, np, nrow, tw, n1, T1, s);
  }
}

// ---------------------------------------------------------------- pair density stage B
// T2[pl][o1][o2][j3] = sum_j2 T1[pl][o1][j2][j3] exp(-2 pi i g2 j2 / N2), g2 = g2lo + o2
// (also used transposed by the adjoint: input axis length N2 -> output axis length n2)
template <typename T, int NO, int PF>
__global__ void __launch_bounds__(256) pd_stageB_kernel(const c2<T>* __restrict__ T1, c2<T>* __restrict__ T2,
                                                        int64_t rows, int N2, int N3,
                                                        const c2<T>* __restrict__ twg, int n2) {
  extern __shared__ unsigned char smem_raw[];
  c2<T>* tw = reinterpret_cast<c2<T>*>(smem_raw);
  const int nchunk = (n2 + TS - 1) / TS;
  for (int oc = 0; oc < nchunk; ++oc) {
    const int o0 = oc * TS;
    const int nout = min(NO, n2 - o0);
    if (oc) __syncthreads();
    load_twiddle_matrix<T>(tw, twg + (int64_t)oc * N2 * TS, N2 * TS);
    const int64_t total = rows * N3;
    for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
      const int j3 = (int)(id % N3);
      const int64_t r = id / N3;  // (pl, o1)
      const c2<T>* src = T1 + r * (int64_t)N2 * N3 + j3;
      c2<T> acc[NO];
#pragma unroll
      for (int t = 0; t < NO; ++t) acc[t] = mk<T>(0, 0);
      if constexpr (PF > 1) {
        c2<T>* my = reinterpret_cast<c2<T>*>(smem_raw + ring_offset<T>(N2)) + threadIdx.x;
#pragma unroll
        for (int j = 0; j < PF - 1; ++j) {
          if (j < N2) cp_async_elem<T>(my + j * RING_THREADS, src + (int64_t)j * N3);
          cp_async_commit();
        }
        for (int j2 = 0; j2 < N2; ++j2) {
          const int jn = j2 + PF - 1;
          if (jn < N2) cp_async_elem<T>(my + (jn % PF) * RING_THREADS, src + (int64_t)jn * N3);
          cp_async_commit();
          cp_async_wait<PF - 1>();  // the group of slice j2 has landed
          const c2<T> x = my[(j2 % PF) * RING_THREADS];
          const c2<T>* twj = tw + j2 * TS;
#pragma unroll
          for (int t = 0; t < NO; ++t) cmac<T>(acc[t], x, twj[t]);
        }
      } else {
        c2<T> nxt = src[0];
        for (int j2 = 0; j2 < N2; ++j2) {
          const c2<T> x = nxt;
          if (j2 + 1 < N2) nxt = src[(int64_t)(j2 + 1) * N3];
          const c2<T>* twj = tw + j2 * TS;
#pragma unroll
          for (int t = 0; t < NO; ++t) cmac<T>(acc[t], x, twj[t]);
        }
      }
      c2<T>* dst = T2 + (r * n2 + o0) * N3 + j3;
#pragma unroll
      for (int t = 0; t < NO; ++t)
        if (t < nout) dst[(int64_t)t * N3] = acc[t];
    }
  }
}

template <typename T, int NO, int PF>
static cudaError_t launch_stageB_pf(const c2<T>* T1, c2<T>* T2, int64_t rows, int N2, int N3, const c2<T>* tw, int n2,
                                    cudaStream_t s) {
  const int smem = PF > 1 ? ring_offset<T>(N2) + PF * RING_THREADS * (int)sizeof(c2<T>) : N2 * TS * (int)sizeof(c2<T>);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(pd_stageB_kernel<T, NO, PF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  pd_stageB_kernel<T, NO, PF><<<grid_for(rows * N3, 256), 256, smem, s>>>(T1, T2, rows, N2, N3, tw, n2);
  return cudaGetLastError();
}

template <typename T, int NO>
static cudaError_t launch_stageB_no(const c2<T>* T1, c2<T>* T2, int64_t rows, int N2, int N3, const c2<T>* tw, int n2,
                                    cudaStream_t s) {
  if (ring_offset<T>(N2) <= 160 * 1024) return launch_stageB_pf<T, NO, RING_PF>(T1, T2, rows, N2, N3, tw, n2, s);
  return launch_stageB_pf<T, NO, 1>(T1, T2, rows, N2, N3, tw, n2, s);
}

template <typename T>
cudaError_t launch_pd_stageB(const c2<T>* T1, c2<T>* T2, int np, int n1, int N2, int N3, const c2<T>* tw, int n2,
                             cudaStream_t s) {
  const int64_t rows = (int64_t)np * n1;
  if (rows == 0) return cudaSuccess;
  switch (width_for(n2)) {
    case 8: return launch_stageB_no<T, 8>(T1, T2, rows, N2, N3, tw, n2, s);
    case 12: return launch_stageB_no<T, 12>(T1, T2, rows, N2, N3, tw, n2, s);
    case 14: return launch_stageB_no<T, 14>(T1, T2, rows, N2, N3, tw, n2, s);
    default: return launch_stageB_no<T, 16>(T1, T2, rows, N2, N3, tw, n2, s);
  }
}

// ---------------------------------------------------------------- factorised pruned DFT (stages A and B)
// With N = r L, j = r m + j' (m < L, j' < r) and outputs g = lo + t (t < n):
//   y_g = sum_j' w_N^(g j') sum_m x_(r m + j') w_L^(g m),   w_N = exp(-2 pi i / N),
// and w_L^(g m) depends on g only through g mod L.  Per residue j' a thread
// forms S_k' = sum_m x_(r m + j') w_L^((b + k') m) for the L classes
// k' = 0..L-1 (b = lo mod L, so output t uses class t mod L, a compile-time
// index), then adds w_N^(g j') S_(t mod L) into output t: N L + r n complex
// multiply-adds per line instead of N n.  Table layout (FP64-accurate,
// stored in T): [m][k'] = w_L^((b + k') m) for m, k' < L, then
// [j'][t] = w_N^((lo + t) j') with a row stride of TS.
template <typename T>
__global__ void twiddle_factored_kernel(c2<T>* __restrict__ tw, int N, int L, int lo, int n) {
  const int r = N / L;
  const int b = pmod(lo, L);
  const int total = L * L + r * TS;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    int t;
    bool on = true;
    if (e < L * L) {
      const int m = e / L, k = e % L;
      t = pmod(-(int64_t)(b + k) * m, L) * r;  // w_L^x = w_N^(x r)
    } else {
      const int jr = (e - L * L) / TS, o = (e - L * L) % TS;
      on = o < n;
      t = pmod(-(int64_t)(lo + o) * jr, N);
    }
    double sn = 0.0, cs = 0.0;
    if (on) sincospi(2.0 * (double)t / (double)N, &sn, &cs);
    tw[e] = mk<T>((T)cs, (T)sn);
  }
}

// The divisor L of N (3, 4, 5, 6 or 8) that minimises N L + (N / L) n, or 0 when the
// factorised form saves less than a fifth of the direct N n.
int factored_radix(int N, int n) {
  int best = 0;
  int64_t cost = (int64_t)N * n * 4 / 5;
  for (int L : {3, 4, 5, 6, 8}) {
    if (N % L || L > n) continue;
    const int64_t c = (int64_t)N * L + (int64_t)(N / L) * n;
    if (c < cost) {
      cost = c;
      best = L;
    }
  }
  return best;
}

template <typename T>
cudaError_t launch_twiddle_factored(c2<T>* tw, int N, int L, int lo, int n, cudaStream_t s) {
  if (L < 2 || N % L || n > TS) return cudaErrorInvalidValue;
  const int total = L * L + (N / L) * TS;
  twiddle_factored_kernel<T><<<(total + 255) / 256, 256, 0, s>>>(tw, N, L, lo, n);
  return cudaGetLastError();
}
template <typename T>
__host__ __device__ constexpr int factored_table(int N, int L) {
  return L * L + (N / L) * TS;
}

// Stage A in the factorised form: as pd_stageA_kernel (PP pairs per thread,
// per-thread cp.async ring of PF slices), with the slices of a line streamed
// residue by residue (slice s is j1 = r (s mod L) + s / L).
template <typename T, int NO, int PP, int L>
__global__ void __launch_bounds__(256) pd_stageA_fact_kernel(const c2<T>* __restrict__ Uk, const c2<T>* __restrict__ Ukp,
                                                             int64_t Nr, int N1, int N23, const int* __restrict__ Lidx,
                                                             const int* __restrict__ Ridx, int nR, int64_t p0, int np,
                                                             int nrow, const c2<T>* __restrict__ twg, int n1,
                                                             c2<T>* __restrict__ T1) {
  constexpr int PF = RING_PF;
  extern __shared__ unsigned char smem_raw[];
  c2<T>* tw = reinterpret_cast<c2<T>*>(smem_raw);
  const int r = N1 / L;
  load_twiddle_matrix<T>(tw, twg, factored_table<T>(N1, L));
  const c2<T>* wl = tw;           // [m][k']
  const c2<T>* wr = tw + L * L;   // [j'][t], stride TS
  const int ngrp = (np + PP - 1) / PP;
  const int64_t total = (int64_t)ngrp * N23;
  c2<T>* my = reinterpret_cast<c2<T>*>(smem_raw + ring_offset<T>((factored_table<T>(N1, L) + TS - 1) / TS)) +
              threadIdx.x;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int j23 = (int)(id % N23);
    const int grp = (int)(id / N23);
    const c2<T>* un[PP];
    const c2<T>* um[PP];
#pragma unroll
    for (int q = 0; q < PP; ++q) {
      const int pl = min(grp * PP + q, np - 1);
      const int64_t p = chunk_pair(pl, p0, nrow, nR);
      un[q] = Uk + (int64_t)Lidx[p / nR] * Nr + j23;
      um[q] = Ukp + (int64_t)Ridx[p % nR] * Nr + j23;
    }
    c2<T> acc[PP][NO], sk[PP][L];
#pragma unroll
    for (int q = 0; q < PP; ++q) {
#pragma unroll
      for (int t = 0; t < NO; ++t) acc[q][t] = mk<T>(0, 0);
#pragma unroll
      for (int k = 0; k < L; ++k) sk[q][k] = mk<T>(0, 0);
    }
    // rows-fastest chunks give a thread's pairs one unoccupied band: its grid
    // is then fetched once per slice for all of them
    bool one_m = true;
#pragma unroll
    for (int q = 1; q < PP; ++q) one_m = one_m && um[q] == um[0];
    auto issue = [&](int sl) {
      const int st = sl % PF;
      const int64_t j = (int64_t)((sl % L) * r + sl / L) * N23;
#pragma unroll
      for (int q = 0; q < PP; ++q) {
        cp_async_elem<T>(my + (st * 2 * PP + 2 * q) * RING_THREADS, un[q] + j);
        if (q == 0 || !one_m) cp_async_elem<T>(my + (st * 2 * PP + 2 * q + 1) * RING_THREADS, um[q] + j);
      }
    };
#pragma unroll
    for (int sl = 0; sl < PF - 1; ++sl) {
      if (sl < N1) issue(sl);
      cp_async_commit();
    }
    for (int jr = 0; jr < r; ++jr) {
#pragma unroll
      for (int m = 0; m < L; ++m) {
        const int sl = jr * L + m;
        if (sl + PF - 1 < N1) issue(sl + PF - 1);
        cp_async_commit();
        cp_async_wait<PF - 1>();  // the group of slice sl has landed
        const int st = sl % PF;
#pragma unroll
        for (int q = 0; q < PP; ++q) {
          const int qm = one_m ? 0 : q;
          const c2<T> x =
              cj_mul<T>(my[(st * 2 * PP + 2 * q) * RING_THREADS], my[(st * 2 * PP + 2 * qm + 1) * RING_THREADS]);
#pragma unroll
          for (int k = 0; k < L; ++k) cmac<T>(sk[q][k], x, wl[m * L + k]);
        }
      }
      const c2<T>* wj = wr + jr * TS;
#pragma unroll
      for (int t = 0; t < NO; ++t) {
        const c2<T> f = wj[t];
#pragma unroll
        for (int q = 0; q < PP; ++q) cmac<T>(acc[q][t], sk[q][t % L], f);
      }
#pragma unroll
      for (int q = 0; q < PP; ++q)
#pragma unroll
        for (int k = 0; k < L; ++k) sk[q][k] = mk<T>(0, 0);
    }
#pragma unroll
    for (int q = 0; q < PP; ++q) {
      const int pl = grp * PP + q;
      if (pl < np) {
        c2<T>* dst = T1 + (int64_t)pl * n1 * N23 + j23;
#pragma unroll
        for (int t = 0; t < NO; ++t)
          if (t < n1) dst[(int64_t)t * N23] = acc[q][t];
      }
    }
  }
}

// Stage B in the factorised form (one row (pl, o1) and j3 per thread).
template <typename T, int NO, int L>
__global__ void __launch_bounds__(256) pd_stageB_fact_kernel(const c2<T>* __restrict__ T1, c2<T>* __restrict__ T2,
                                                             int64_t rows, int N2, int N3,
                                                             const c2<T>* __restrict__ twg, int n2) {
  constexpr int PF = RING_PF;
  extern __shared__ unsigned char smem_raw[];
  c2<T>* tw = reinterpret_cast<c2<T>*>(smem_raw);
  const int r = N2 / L;
  load_twiddle_matrix<T>(tw, twg, factored_table<T>(N2, L));
  const c2<T>* wl = tw;
  const c2<T>* wr = tw + L * L;
  c2<T>* my = reinterpret_cast<c2<T>*>(smem_raw + ring_offset<T>((factored_table<T>(N2, L) + TS - 1) / TS)) +
              threadIdx.x;
  const int64_t total = rows * N3;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int j3 = (int)(id % N3);
    const int64_t row = id / N3;  // (pl, o1)
    const c2<T>* src = T1 + row * (int64_t)N2 * N3 + j3;
    c2<T> acc[NO], sk[L];
#pragma unroll
    for (int t = 0; t < NO; ++t) acc[t] = mk<T>(0, 0);
#pragma unroll
    for (int k = 0; k < L; ++k) sk[k] = mk<T>(0, 0);
#pragma unroll
    for (int sl = 0; sl < PF - 1; ++sl) {
      if (sl < N2) cp_async_elem<T>(my + sl * RING_THREADS, src + (int64_t)((sl % L) * r + sl / L) * N3);
      cp_async_commit();
    }
    for (int jr = 0; jr < r; ++jr) {
#pragma unroll
      for (int m = 0; m < L; ++m) {
        const int sl = jr * L + m;
        const int sn = sl + PF - 1;
        if (sn < N2) cp_async_elem<T>(my + (sn % PF) * RING_THREADS, src + (int64_t)((sn % L) * r + sn / L) * N3);
        cp_async_commit();
        cp_async_wait<PF - 1>();
        const c2<T> x = my[(sl % PF) * RING_THREADS];
#pragma unroll
        for (int k = 0; k < L; ++k) cmac<T>(sk[k], x, wl[m * L + k]);
      }
      const c2<T>* wj = wr + jr * TS;
#pragma unroll
      for (int t = 0; t < NO; ++t) cmac<T>(acc[t], sk[t % L], wj[t]);
#pragma unroll
      for (int k = 0; k < L; ++k) sk[k] = mk<T>(0, 0);
    }
    c2<T>* dst = T2 + (row * n2) * N3 + j3;
#pragma unroll
    for (int t = 0; t < NO; ++t)
      if (t < n2) dst[(int64_t)t * N3] = acc[t];
  }
}

template <typename T, int NO, int L>
static cudaError_t launch_stageA_fact_l(const c2<T>* Uk, const c2<T>* Ukp, int64_t Nr, int N1, int N23,
                                        const int* Lidx, const int* Ridx, int nR, int64_t p0, int np, int nrow,
                                        const c2<T>* twf, int n1, c2<T>* T1, cudaStream_t s) {
  constexpr int PP = sizeof(T) == 4 ? 2 : 1;
  const int64_t total = (int64_t)((np + PP - 1) / PP) * N23;
  if (total == 0) return cudaSuccess;
  const int smem = ring_offset<T>((factored_table<T>(N1, L) + TS - 1) / TS) +
                   RING_PF * 2 * PP * RING_THREADS * (int)sizeof(c2<T>);
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(pd_stageA_fact_kernel<T, NO, PP, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  pd_stageA_fact_kernel<T, NO, PP, L><<<grid_for(total, 256), 256, smem, s>>>(Uk, Ukp, Nr, N1, N23, Lidx, Ridx, nR,
                                                                             p0, np, nrow, twf, n1, T1);
  return cudaGetLastError();
}

template <typename T, int NO>
static cudaError_t launch_stageA_fact_no(const c2<T>* Uk, const c2<T>* Ukp, int64_t Nr, int N1, int N23,
                                         const int* Lidx, const int* Ridx, int nR, int64_t p0, int np, int nrow,
                                         const c2<T>* twf, int L, int n1, c2<T>* T1, cudaStream_t s) {
  switch (L) {
    case 3: return launch_stageA_fact_l<T, NO, 3>(Uk, Ukp, Nr, N1, N23, Lidx, Ridx, nR, p0, np, nrow, twf, n1, T1, s);
    case 4: return launch_stageA_fact_l<T, NO, 4>(Uk, Ukp, Nr, N1, N23, Lidx, Ridx, nR, p0, np, nrow, twf, n1, T1, s);
    case 5: return launch_stageA_fact_l<T, NO, 5>(Uk, Ukp, Nr, N1, N23, Lidx, Ridx, nR, p0, np, nrow, twf, n1, T1, s);
    case 6: return launch_stageA_fact_l<T, NO, 6>(Uk, Ukp, Nr, N1, N23, Lidx, Ridx, nR, p0, np, nrow, twf, n1, T1, s);
    case 8: return launch_stageA_fact_l<T, NO, 8>(Uk, Ukp, Nr, N1, N23, Lidx, Ridx, nR, p0, np, nrow, twf, n1, T1, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_pd_stageA_fact(const c2<T>* Uk, const c2<T>* Ukp, int64_t Nr, int N1, int N23, const int* Lidx,
                                  const int* Ridx, int nR, int64_t p0, int np, int nrow, const c2<T>* twf, int L,
                                  int n1, c2<T>* T1, cudaStream_t s) {
  if (n1 > TS || L < 2 || N1 % L || nrow < 1 || np % nrow) return cudaErrorInvalidValue;
  switch (width_for(n1)) {
    case 8: return launch_stageA_fact_no<T, 8>(Uk, Ukp, Nr, N1, N23, Lidx, Ridx, nR, p0, np, nrow, twf, L, n1, T1, s);
    case 12: return launch_stageA_fact_no<T, 12>(Uk, Ukp, Nr, N1, N23, Lidx, Ridx, nR, p0, np, nrow, twf, L, n1, T1, s);
    case 14: return launch_stageA_fact_no<T, 14>(Uk, Ukp, Nr, N1, N23, Lidx, Ridx, nR, p0, np, nrow, twf, L, n1, T1, s);
    default: return launch_stageA_fact_no<T, 16>(Uk, Ukp, Nr, N1, N23, Lidx, Ridx, nR, p0, np, nrow, twf, L, n1, T1, s);
  }
}

template <typename T, int NO, int L>
static cudaError_t launch_stageB_fact_l(const c2<T>* T1, c2<T>* T2, int64_t rows, int N2, int N3, const c2<T>* twf,
                                        int n2, cudaStream_t s) {
  const int smem =
      ring_offset<T>((factored_table<T>(N2, L) + TS - 1) / TS) + RING_PF * RING_THREADS * (int)sizeof(c2<T>);
  pd_stageB_fact_kernel<T, NO, L><<<grid_for(rows * N3, 256), 256, smem, s>>>(T1, T2, rows, N2, N3, twf, n2);
  return cudaGetLastError();
}

template <typename T, int NO>
static cudaError_t launch_stageB_fact_no(const c2<T>* T1, c2<T>* T2, int64_t rows, int N2, int N3, const c2<T>* twf,
                                         int L, int n2, cudaStream_t s) {
  switch (L) {
    case 3: return launch_stageB_fact_l<T, NO, 3>(T1, T2, rows, N2, N3, twf, n2, s);
    case 4: return launch_stageB_fact_l<T, NO, 4>(T1, T2, rows, N2, N3, twf, n2, s);
    case 5: return launch_stageB_fact_l<T, NO, 5>(T1, T2, rows, N2, N3, twf, n2, s);
    case 6: return launch_stageB_fact_l<T, NO, 6>(T1, T2, rows, N2, N3, twf, n2, s);
    case 8: return launch_stageB_fact_l<T, NO, 8>(T1, T2, rows, N2, N3, twf, n2, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_pd_stageB_fact(const c2<T>* T1, c2<T>* T2, int np, int n1, int N2, int N3, const c2<T>* twf, int L,
                                  int n2, cudaStream_t s) {
  const int64_t rows = (int64_t)np * n1;
  if (rows == 0) return cudaSuccess;
  if (n2 > TS || L < 2 || N2 % L) return cudaErrorInvalidValue;
  switch (width_for(n2)) {
    case 8: return launch_stageB_fact_no<T, 8>(T1, T2, rows, N2, N3, twf, L, n2, s);
    case 12: return launch_stageB_fact_no<T, 12>(T1, T2, rows, N2, N3, twf, L, n2, s);
    case 14: return launch_stageB_fact_no<T, 14>(T1, T2, rows, N2, N3, twf, L, n2, s);
    default: return launch_stageB_fact_no<T, 16>(T1, T2, rows, N2, N3, twf, L, n2, s);
  }
}

// ---------------------------------------------------------------- pair density stage C
template <typename T>
__global__ void __launch_bounds__(256) pd_stageC_kernel(const c2<T>* __restrict__ T2, int np, int n1, int n2, int N3,
                                                        const int* __restrict__ gfft, int NG, int g1lo, int g2lo,
                                                        double inv_nr, int64_t p0, int nrow, int nR,
                                                        const c2<T>* __restrict__ twg, c2<T>* __restrict__ Nout) {
  // Each thread handles one G and PG consecutive pairs (the fastest-axis DFT
  // of each pair; PG independent loads per step).
  constexpr int PG = 4;
  extern __shared__ unsigned char smem_raw[];
  c2<T>* tw = reinterpret_cast<c2<T>*>(smem_raw);
  if (twg) {
    // the table of twiddle_line_kernel (the same values fill_twiddles forms)
    for (int t = threadIdx.x; t < N3; t += blockDim.x) tw[t] = twg[t];
    __syncthreads();
  } else {
    fill_twiddles<T>(tw, N3);
  }
  const int ngrp = (np + PG - 1) / PG;
  const int64_t total = (int64_t)ngrp * NG;
  const T scale = (T)inv_nr;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int ig = (int)(id % NG);
    const int grp = (int)(id / NG);
    const int g1 = gfft[3 * ig], g2 = gfft[3 * ig + 1], g3 = gfft[3 * ig + 2];
    const int step = pmod(-(int64_t)g3, N3);
    c2<T> acc[PG];
    int64_t pidx[PG];
    const c2<T>* src[PG];
#pragma unroll
    for (int q = 0; q < PG; ++q) {
      const int pl = min(grp * PG + q, np - 1);
      pidx[q] = chunk_pair(pl, p0, nrow, nR);
      src[q] = T2 + (((int64_t)pl * n1 + (g1 - g1lo)) * n2 + (g2 - g2lo)) * N3;
      acc[q] = mk<T>(0, 0);
    }
    // the PG pairs advance together, UJ steps at a time: PG x UJ independent
    // loads are in flight before their multiply-adds (the reads of the
    // stage-B output are strided, so their latency, not issue, is the limit)
    constexpr int UJ = 4;
    int idx = 0;
    int j3 = 0;
    for (; j3 + UJ <= N3; j3 += UJ) {
      c2<T> x[UJ][PG], f[UJ];
#pragma unroll
      for (int u = 0; u < UJ; ++u) {
#pragma unroll
        for (int q = 0; q < PG; ++q) x[u][q] = src[q][j3 + u];
        f[u] = tw[idx];
        idx += step;
        if (idx >= N3) idx -= N3;
      }
#pragma unroll
      for (int u = 0; u < UJ; ++u)
#pragma unroll
        for (int q = 0; q < PG; ++q) cmac<T>(acc[q], x[u][q], f[u]);
    }
    for (; j3 < N3; ++j3) {
      const c2<T> f = tw[idx];
#pragma unroll
      for (int q = 0; q < PG; ++q) cmac<T>(acc[q], src[q][j3], f);
      idx += step;
      if (idx >= N3) idx -= N3;
    }
#pragma unroll
    for (int q = 0; q < PG; ++q)
      if (grp * PG + q < np) Nout[pidx[q] * NG + ig] = mk<T>(acc[q].x * scale, acc[q].y * scale);
  }
}

// ---------------------------------------------------------------- pair density stages B + C fused
// One block per (pair, slab of OB first-axis outputs o1): the middle-axis DFT
// of the slab goes to shared memory,
//   T2[o1][o2][j3] = sum_j2 T1[pl][o1][j2][j3] exp(-2 pi i g2 j2 / N2),
// and the fastest axis is then evaluated on the sphere points whose g1 lies in
// the slab (a contiguous range of the Miller-ordered sphere, g1start),
//   N[p][G] = (1/N_r) sum_j3 T2[o1(G)][o2(G)][j3] exp(-2 pi i g3 j3 / N3),
// written along G.  Same products in the same order as stage B followed by
// stage C (bit-identical), without the global round trip of T2 and with the
// fastest-axis lines read from shared memory.
template <typename T, int NO>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) pd_stageBC_kernel(const c2<T>* __restrict__ T1, int np, int n1, int N2, int N3,
                                                         const c2<T>* __restrict__ twg, int n2,
                                                         const int* __restrict__ gfft,
                                                         const int* __restrict__ g1start, int OB, int NG, int g1lo,
                                                         int g2lo, double inv_nr, int64_t p0,
                                                         c2<T>* __restrict__ Nout) {
  extern __shared__ unsigned char smem_raw[];
  c2<T>* tw2 = reinterpret_cast<c2<T>*>(smem_raw);  // [N2][TS], outputs o2 < n2 <= NO
  c2<T>* tw3 = tw2 + N2 * TS;                         // exp(2 pi i t / N3)
  c2<T>* T2s = tw3 + N3;                              // [OB][n2][N3]
  for (int e = threadIdx.x; e < N2 * TS; e += blockDim.x) tw2[e] = twg[e];
  fill_twiddles<T>(tw3, N3);  // ends with a block barrier
  const int nslab = (n1 + OB - 1) / OB;
  const T scale = (T)inv_nr;
  for (int64_t item = blockIdx.x; item < (int64_t)np * nslab; item += gridDim.x) {
    const int pl = (int)(item / nslab);
    const int o1a = (int)(item % nslab) * OB;
    const int ob = min(OB, n1 - o1a);
    for (int cidx = threadIdx.x; cidx < ob * N3; cidx += blockDim.x) {
      const int r = cidx / N3, j3 = cidx % N3;
      const c2<T>* src = T1 + ((int64_t)pl * n1 + o1a + r) * N2 * N3 + j3;
      c2<T> acc[NO];
#pragma unroll
      for (int t = 0; t < NO; ++t) acc[t] = mk<T>(0, 0);
      // the middle-axis line in slices of 4: four independent loads in
      // flight before their multiply-adds (the line is strided by N3); in
      // FP32 at most 64 registers, so two 512-thread blocks fit on an SM
      for (int jb = 0; jb < N2; jb += 4) {
        c2<T> x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = jb + u < N2 ? src[(int64_t)(jb + u) * N3] : mk<T>(0, 0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (jb + u < N2) {
            const c2<T>* twj = tw2 + (jb + u) * TS;
#pragma unroll
            for (int t = 0; t < NO; ++t) cmac<T>(acc[t], x[u], twj[t]);
          }
        }
      }
      c2<T>* dst = T2s + (int64_t)r * n2 * N3 + j3;
#pragma unroll
      for (int t = 0; t < NO; ++t)
        if (t < n2) dst[(int64_t)t * N3] = acc[t];
    }
    __syncthreads();
    const int gs = g1start[o1a], ge = g1start[o1a + ob];
    for (int ig = gs + threadIdx.x; ig < ge; ig += blockDim.x) {
      const int g1 = gfft[3 * ig], g2 = gfft[3 * ig + 1], g3 = gfft[3 * ig + 2];
      const c2<T>* line = T2s + ((int64_t)(g1 - g1lo - o1a) * n2 + (g2 - g2lo)) * N3;
      const int step = pmod(-(int64_t)g3, N3);
      c2<T> acc = mk<T>(0, 0);
      int idx = 0;
      for (int j3 = 0; j3 < N3; ++j3) {
        cmac<T>(acc, line[j3], tw3[idx]);
        idx += step;
        if (idx >= N3) idx -= N3;
      }
      Nout[(p0 + pl) * NG + ig] = mk<T>(acc.x * scale, acc.y * scale);
    }
    __syncthreads();
  }
}

// g1start[o] = the first sphere point with g1 - g1lo >= o, o in [0, n1]
// (the sphere is sorted by g1; binary search per o).
__global__ void g1start_kernel(const int* __restrict__ gfft, int NG, int g1lo, int n1, int* __restrict__ out) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o <= n1; o += gridDim.x * blockDim.x) {
    int lo = 0, hi = NG;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (gfft[3 * mid] - g1lo < o) lo = mid + 1;
      else hi = mid;
    }
    out[o] = lo;
  }
}

cudaError_t launch_g1start(const int* gfft, int NG, int g1lo, int n1, int* out, cudaStream_t s) {
  g1start_kernel<<<(n1 + 1 + 127) / 128, 128, 0, s>>>(gfft, NG, g1lo, n1, out);
  return cudaGetLastError();
}

// Slab height OB of the fused kernel: the largest that keeps its shared
// memory within 48 KB (0 if even one first-axis output does not fit, or the
// middle axis has more than 16 outputs).
template <typename T>
int pd_stageBC_slab(int n1, int n2, int N2, int N3) {
  if (n2 > TS) return 0;
  const int64_t fixed = ((int64_t)N2 * TS + N3) * (int64_t)sizeof(c2<T>);
  const int64_t per = (int64_t)n2 * N3 * (int64_t)sizeof(c2<T>);
  const int64_t room = 48 * 1024 - fixed;
  if (room < per) return 0;
  return (int)std::min<int64_t>(n1, room / per);
}

template <typename T, int NO>
static cudaError_t launch_stageBC_no(const c2<T>* T1, int np, int n1, int N2, int N3, const c2<T>* tw, int n2,
                                     const int* gfft, const int* g1start, int OB, int NG, int g1lo, int g2lo,
                                     double inv_nr, int64_t p0, c2<T>* Nout, cudaStream_t s) {
  const int nslab = (n1 + OB - 1) / OB;
  const int64_t items = (int64_t)np * nslab;
  const int threads = (int)std::min<int64_t>(512, std::max<int64_t>(64, ((int64_t)OB * N3 + 31) / 32 * 32));
  const size_t smem = ((size_t)N2 * TS + N3 + (size_t)OB * n2 * N3) * sizeof(c2<T>);
  const int blocks = (int)std::min<int64_t>(items, 152 * 16);
  pd_stageBC_kernel<T, NO><<<blocks, threads, smem, s>>>(T1, np, n1, N2, N3, tw, n2, gfft, g1start, OB, NG, g1lo, g2lo,
                                                         inv_nr, p0, Nout);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pd_stageBC(const c2<T>* T1, int np, int n1, int N2, int N3, const c2<T>* tw, int n2,
                              const int* gfft, const int* g1start, int OB, int NG, int g1lo, int g2lo, double inv_nr,
                              int64_t p0, c2<T>* Nout, cudaStream_t s) {
  if (np == 0 || OB < 1) return cudaSuccess;
  switch (width_for(n2)) {
    case 8: return launch_stageBC_no<T, 8>(T1, np, n1, N2, N3, tw, n2, gfft, g1start, OB, NG, g1lo, g2lo, inv_nr, p0, Nout, s);
    case 12: return launch_stageBC_no<T, 12>(T1, np, n1, N2, N3, tw, n2, gfft, g1start, OB, NG, g1lo, g2lo, inv_nr, p0, Nout, s);
    case 14: return launch_stageBC_no<T, 14>(T1, np, n1, N2, N3, tw, n2, gfft, g1start, OB, NG, g1lo, g2lo, inv_nr, p0, Nout, s);
    default: return launch_stageBC_no<T, 16>(T1, np, n1, N2, N3, tw, n2, gfft, g1start, OB, NG, g1lo, g2lo, inv_nr, p0, Nout, s);
  }
}

// ---------------------------------------------------------------- PAW term (Eq. 6, steps 8-9)
// N[(a nR + b) NG + g] += sum_kp Pm[b][kp] R[a][kp][g] for every occupied row a
// of the block: one complex GEMM (nR x KP) x (KP x NG) per a, 64 x 64 tiles,
// 4 x 4 outputs a thread.
constexpr int PWT = 64, PWK = 16;

template <typename T>
__global__ void __launch_bounds__(256) paw_gemm_kernel(const c2<T>* __restrict__ R, const c2<T>* __restrict__ Pm,
                                                       int KP, int nR, int NG, c2<T>* __restrict__ N) {
  __shared__ c2<T> As[PWK][PWT];
  __shared__ c2<T> Bs[PWK][PWT];
  const int a = blockIdx.z;
  const int b0 = blockIdx.y * PWT, g0 = blockIdx.x * PWT;
  const c2<T>* Ra = R + (int64_t)a * KP * NG;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  c2<T> acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = mk<T>(0, 0);
  for (int k0 = 0; k0 < KP; k0 += PWK) {
#pragma unroll
    for (int q = 0; q < (PWK * PWT) / 256; ++q) {
      const int e = threadIdx.x + 256 * q;
      {
        const int r = e / PWK, kk = e % PWK;
        As[kk][r] = (b0 + r < nR && k0 + kk < KP) ? Pm[(int64_t)(b0 + r) * KP + k0 + kk] : mk<T>(0, 0);
      }
      {
        const int kk = e / PWT, c = e % PWT;
        Bs[kk][c] = (k0 + kk < KP && g0 + c < NG) ? Ra[(int64_t)(k0 + kk) * NG + g0 + c] : mk<T>(0, 0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < PWK; ++kk) {
      c2<T> x[4], y[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) x[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) y[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) cmac<T>(acc[r][c], x[r], y[c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int b = b0 + ty + 16 * r, g = g0 + tx + 16 * c;
      if (b < nR && g < NG) {
        c2<T>* p = N + ((int64_t)a * nR + b) * NG + g;
        c2<T> v = *p;
        v.x += acc[r][c].x;
        v.y += acc[r][c].y;
        *p = v;
      }
    }
}

template <typename T>
cudaError_t launch_paw_gemm(const c2<T>* R, const c2<T>* Pm, int KP, int nL, int nR, int NG, c2<T>* N,
                            cudaStream_t s) {
  if (KP == 0 || nL == 0 || nR == 0 || NG == 0) return cudaSuccess;
  dim3 grid((NG + PWT - 1) / PWT, (nR + PWT - 1) / PWT, nL);
  paw_gemm_kernel<T><<<grid, 256, 0, s>>>(R, Pm, KP, nR, NG, N);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pd_stageC(const c2<T>* T2, int np, int n1, int n2, int N3, const int* gfft, int NG, int g1lo,
                             int g2lo, double inv_nr, int64_t p0, int nrow, int nR, const c2<T>* tw3, c2<T>* Nout,
                             cudaStream_t s) {
  const int64_t total = (int64_t)((np + 3) / 4) * NG;
  if (total == 0) return cudaSuccess;
  if (nrow < 1 || np % nrow) return cudaErrorInvalidValue;
  pd_stageC_kernel<T><<<grid_for(total, 256), 256, N3 * sizeof(c2<T>), s>>>(T2, np, n1, n2, N3, gfft, NG, g1lo, g2lo,
                                                                          inv_nr, p0, nrow, nR, tw3, Nout);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- PAW factor (FP64)
template <typename T>
__global__ void paw_R_kernel(const double2* __restrict__ Pk, int KP, const int* __restrict__ Lidx, int nL,
                             const double2* __restrict__ Q, const int* __restrict__ atom_of_kp,
                             const int* __restrict__ idx_in_atom, const int* __restrict__ atom_off,
                             const int64_t* __restrict__ q_off, const int* __restrict__ nproj, int NG,
                             c2<T>* __restrict__ R) {
  const int64_t total = (int64_t)nL * KP * NG;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int ig = (int)(id % NG);
    int64_t r = id / NG;
    const int kp = (int)(r % KP);
    const int a = (int)(r / KP);
    const int atom = atom_of_kp[kp];
    const int j = idx_in_atom[kp];
    const int ni = nproj[atom];
    const double2* pn = Pk + (int64_t)Lidx[a] * KP + atom_off[atom];
    const double2* qa = Q + q_off[atom] + (int64_t)j * NG + ig;
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < ni; ++i) {
      // conj(P_ni) * Q_ij(G)
      const double2 p = pn[i];
      const double2 q = qa[(int64_t)i * ni * NG];
      acc.x = fma(p.x, q.x, acc.x);
      acc.x = fma(p.y, q.y, acc.x);
      acc.y = fma(p.x, q.y, acc.y);
      acc.y = fma(-p.y, q.x, acc.y);
    }
    R[id] = mk<T>((T)acc.x, (T)acc.y);
  }
}

template <typename T>
cudaError_t launch_paw_R(const double2* Pk, int KP, const int* Lidx, int nL, const double2* Q, const int* atom_of_kp,
                         const int* idx_in_atom, const int* atom_off, const int64_t* q_off, const int* nproj, int NG,
                         c2<T>* R, cudaStream_t s) {
  const int64_t total = (int64_t)nL * KP * NG;
  if (total == 0) return cudaSuccess;
  paw_R_kernel<T><<<grid_for(total, 256), 256, 0, s>>>(Pk, KP, Lidx, nL, Q, atom_of_kp, idx_in_atom, atom_off, q_off,
                                                       nproj, NG, R);
  return cudaGetLastError();
}

template <typename T>
__global__ void gather_P_kernel(const double2* __restrict__ P, int KP, const int* __restrict__ Ridx, int nR,
                                c2<T>* __restrict__ out) {
  const int64_t total = (int64_t)nR * KP;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int kp = (int)(id % KP);
    const int b = (int)(id / KP);
    const double2 v = P[(int64_t)Ridx[b] * KP + kp];
    out[id] = mk<T>((T)v.x, (T)v.y);
  }
}

template <typename T>
cudaError_t launch_gather_P(const double2* P, int KP, const int* Ridx, int nR, c2<T>* out, cudaStream_t s) {
  const int64_t total = (int64_t)nR * KP;
  if (total == 0) return cudaSuccess;
  gather_P_kernel<T><<<grid_for(total, 256), 256, 0, s>>>(P, KP, Ridx, nR, out);
  return cudaGetLastError();
}

__global__ void pair_params_kernel(const double* __restrict__ ek, const double* __restrict__ fk,
                                   const double* __restrict__ ekp, const double* __restrict__ fkp,
                                   const int* __restrict__ Lidx, int nL, const int* __restrict__ Ridx, int nR,
                                   double* __restrict__ d, double* __restrict__ df) {
  const int64_t total = (int64_t)nL * nR;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int n = Lidx[id / nR];
    const int m = Ridx[id % nR];
    d[id] = ek[n] - ekp[m];
    const double x = fk[n] - fkp[m];
    df[id] = x > 0.0 ? x : 0.0;
  }
}

cudaError_t launch_pair_params(const double* ek, const double* fk, const double* ekp, const double* fkp,
                               const int* Lidx, int nL, const int* Ridx, int nR, double* d, double* df,
                               cudaStream_t s) {
  const int64_t total = (int64_t)nL * nR;
  if (total == 0) return cudaSuccess;
  pair_params_kernel<<<grid_for(total, 256), 256, 0, s>>>(ek, fk, ekp, fkp, Lidx, nL, Ridx, nR, d, df);
  return cudaGetLastError();
}

#define RPA_INST(T)                                                                                              \
  template cudaError_t launch_dft_axis<T>(const c2<T>*, c2<T>*, int64_t, int, int, int, int, int, int, int, int, \
                                          cudaStream_t);                                                         \
  template cudaError_t launch_scatter_box<T>(const double2*, int, int, const int*, int64_t, c2<T>*, cudaStream_t); \
  template cudaError_t launch_pd_stageB<T>(const c2<T>*, c2<T>*, int, int, int, int, const c2<T>*, int,          \
                                           cudaStream_t);                                                        \
  template cudaError_t launch_twiddle_matrix<T>(c2<T>*, int, int, int, cudaStream_t);                             \
  template cudaError_t launch_twiddle_factored<T>(c2<T>*, int, int, int, int, cudaStream_t);                    \
  template cudaError_t launch_pd_stageA_fact<T>(const c2<T>*, const c2<T>*, int64_t, int, int, const int*,        \
                                                const int*, int, int64_t, int, int, const c2<T>*, int, int,       \
                                                c2<T>*, cudaStream_t);                                            \
  template cudaError_t launch_pd_stageB_fact<T>(const c2<T>*, c2<T>*, int, int, int, int, const c2<T>*, int, int,  \
                                                cudaStream_t);                                                    \
  template cudaError_t launch_pd_stageA<T>(const c2<T>*, const c2<T>*, int64_t, int, int, const int*, const int*, \
                                           int, int64_t, int, int, const c2<T>*, int, c2<T>*, cudaStream_t);     \
  template cudaError_t launch_pd_stageBC<T>(const c2<T>*, int, int, int, int, const c2<T>*, int, const int*,     \
                                             const int*, int, int, int, int, double, int64_t, c2<T>*, cudaStream_t); \
  template int pd_stageBC_slab<T>(int, int, int, int);                                                            \
  template cudaError_t launch_pd_stageC<T>(const c2<T>*, int, int, int, int, const int*, int, int, int, double,    \
                                           int64_t, int, int, const c2<T>*, c2<T>*, cudaStream_t);              \
  template cudaError_t launch_twiddle_line<T>(c2<T>*, int, cudaStream_t);                                       \
  template cudaError_t launch_paw_gemm<T>(const c2<T>*, const c2<T>*, int, int, int, int, c2<T>*, cudaStream_t); \
  template cudaError_t launch_paw_R<T>(const double2*, int, const int*, int, const double2*, const int*,          \
                                       const int*, const int*, const int64_t*, const int*, int, c2<T>*,          \
                                       cudaStream_t);                                                            \
  template cudaError_t launch_gather_P<T>(const double2*, int, const int*, int, c2<T>*, cudaStream_t);

RPA_INST(float)
RPA_INST(double)

}  // namespace rpa
