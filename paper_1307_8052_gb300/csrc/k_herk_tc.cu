// Tensor-core grouped Hermitian rank-k update of chi0 (Eq. 17, the paper's
// "multi-u" zherk) for every frequency, on the 5th-generation tensor cores.
//
// Real-stacked form.  With a_p = n_p(G_i), b_p = n_p(G_j) and the K index
// k = 2p + c running over (pair, re/im):
//   Re chi_ij = sum_k A_ik X_jk,  Im chi_ij = sum_k A_ik Z_jk,
//   A = w_p(w) (Re a, Im a),  X = (Re b, Im b),  Z = (-Im b, Re b).
// Each operand is split into bfloat16 terms x = x_hi + x_lo (+ x_mid for
// three terms); the products hi*hi + hi*lo + lo*hi (and hi*mid, mid*hi,
// mid*mid, hi*lo2, lo2*hi for three terms) are accumulated in FP32 in tensor
// memory (TMEM) for one fold (64 K-elements by default).  The tensor cores
// truncate while accumulating (measured: the bias of |chi0| grows linearly
// with the fold length), so each fold's partial is added to FP32 running sums
// in registers (round to nearest) and those go to the FP64 chi0 every few
// folds.
//
// Data path: one prep kernel per k-block writes the unweighted X, Z operand
// splits (K-major, bfloat16), one prep kernel writes the weighted A splits for
// all frequencies; the kernel streams 128-row tiles with TMA
// (cp.async.bulk.tensor; 64-element stages with the 128-byte swizzle in a
// 2-stage ring, or 32-element stages with the 64-byte swizzle for three
// terms), one thread issues one tcgen05.mma (M = 128, N = 256, K = 16) per
// product with the X tile stacked on the Z tile, so Re and Im land in one
// 256-column TMEM buffer; two such buffers alternate, and sixteen epilogue
// warps drain one with tcgen05.ld while the MMAs fill the other.  Only
// lower-triangle tiles are launched.  A batched product variant (GEMM = true)
// serves the adjoint and the PAW term.  Every wait is bounded by the GPU
// global timer; on timeout the CTA raises a flag, drains, frees TMEM and exits.
#include "rpa_internal.h"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>

namespace rpa {
namespace tc {

constexpr int BM = 128;               // tile rows (G_i)
constexpr int BN = 128;               // tile cols (G_j)
constexpr int EPI_WARPS = 16;         // epilogue warps: 4 per TMEM lane quarter
constexpr int NUM_THREADS = 64 + 32 * EPI_WARPS;  // warp 0 TMA, warp 1 MMA, warps 2-17 epilogue
constexpr uint64_t TIMEOUT_NS = 4000000000ull;  // 4 s per wait

// Pipeline shapes: BK bf16 K-elements per stage (64: 128-byte rows with the
// 128-byte swizzle; 32: 64-byte rows with the 64-byte swizzle) and STAGES
// stages in the shared-memory ring.
template <int TERMS, int BK_, int STAGES_> struct Cfg {
  static constexpr int BK = BK_;
  static constexpr int STAGES = STAGES_;
  static constexpr int TILE_BYTES = BM * BK * 2;
  static constexpr int A_TILES = TERMS;             // A hi, (mid), lo
  static constexpr int B_TILES = 2 * TERMS;         // per term X then Z: one 256-row B operand
  static constexpr int STAGE_BYTES = (A_TILES + B_TILES) * TILE_BYTES;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false if the timer expired or another role aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (gtimer() - t0 > TIMEOUT_NS) return false;
  }
}

__device__ __forceinline__ bool mbar_wait_timer(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = gtimer();
  while (!mbar_try_wait(bar, parity))
    if (gtimer() - t0 > TIMEOUT_NS) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int k, int row) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(k), "r"(row)
      : "memory");
}

// UMMA shared-memory descriptor of a K-major tile: 8-row core groups of
// 8 * row-bytes; layout code 2 = 128-byte swizzle (BK = 64), 4 = 64-byte (BK = 32).
template <int BK>
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr) {
  constexpr uint32_t row_bytes = BK * 2;
  constexpr uint64_t layout = BK == 64 ? 2 : 4;
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);      // start address (16-byte units)
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)((8 * row_bytes) >> 4) << 32;   // stride byte offset between 8-row groups
  d |= (uint64_t)1 << 46;                        // descriptor version (tcgen05)
  d |= layout << 61;
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tri_tile(int t, int& ti, int& tj) {
  int i = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (i * (i + 1) / 2 > t) --i;
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  ti = i;
  tj = t - i * (i + 1) / 2;
}

struct Maps {
  CUtensorMap a[3];  // weighted A terms (rows = w * NGpad + i)
  CUtensorMap x[3];  // X terms
  CUtensorMap z[3];  // Z terms
};

// Extra arguments of the weighted-product variant (GEMM = true): the adjoint
// of the rank-k update, out[p][g] = 2 sum_w wgt[w][p] sum_k N[p][k] conj(Gam_w[k][g])
// (Eq. 17 transposed).  A holds the pair densities (rows p, shared by all w),
// X / Z the per-frequency Gam (rows w * NGpad + g); K runs over w and k, and
// the weight of row p is applied to every fold as it leaves tensor memory.
// Without weights the variant is a plain batched product
// out_y[p][g] (+)= sum_k A[p][k] conj(B_y[g][k]) over blockIdx.y = y (the PAW
// term of Eq. 6: one batch per occupied band, B_y = conj R_y).
struct GemmArgs {
  int64_t P;          // rows (pairs)
  int nkw;            // K stages per frequency
  int ngt;            // column tiles (NGpad / BN)
  const float* wgt;   // [nw][P], or null: weight 1
  float2* out;        // [P][NG] per batch
  int nwb;            // frequencies per batch: B rows (y * nwb + w) * NGpad + g
  int accumulate;     // add to out instead of writing it
  int64_t out_batch;  // elements between the outputs of consecutive batches
};

template <int TERMS, int BK, int STAGES, bool GEMM>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    herk_tc_kernel(const __grid_constant__ Maps maps, int NG, int NGpad, int nk, int fold, int flush, double2* __restrict__ chi,
                   int* __restrict__ err, const GemmArgs ga) {
  using C = Cfg<TERMS, BK, STAGES>;
  constexpr int TILE_BYTES = C::TILE_BYTES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* mma_done = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = blockIdx.y;  // HERK: frequency; GEMM: batch
  int ti, tj;
  if constexpr (GEMM) {
    ti = blockIdx.x / ga.ngt;  // row tile of pairs
    tj = blockIdx.x % ga.ngt;
  } else {
    tri_tile(blockIdx.x, ti, tj);
  }
  const int i0 = ti * BM, j0 = tj * BN;
  const int nfold = (nk + fold - 1) / fold;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 32 * EPI_WARPS);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        if (kb >= STAGES && !mbar_wait(&empty[s], ((kb / STAGES) & 1) ^ 1, abort_flag)) {
          *abort_flag = 1;
          atomicExch(err, 1);
          break;
        }
        mbar_expect_tx(&full[s], C::STAGE_BYTES);
        unsigned char* st = smem + s * C::STAGE_BYTES;
        // HERK: A rows w * NGpad + i0 (weighted per frequency), X / Z rows j0;
        // GEMM: A rows i0 (pairs), X / Z rows wk * NGpad + j0 of frequency wk
        const int wk = GEMM ? kb / ga.nkw : 0;
        const int k = GEMM ? (kb - wk * ga.nkw) * BK : kb * BK;
        const int arow = GEMM ? i0 : w * NGpad + i0;
        const int brow = GEMM ? (w * ga.nwb + wk) * NGpad + j0 : j0;
#pragma unroll
        for (int t = 0; t < TERMS; ++t) tma_load_2d(st + t * TILE_BYTES, &maps.a[t], &full[s], k, arow);
#pragma unroll
        for (int t = 0; t < TERMS; ++t) {
          tma_load_2d(st + (TERMS + 2 * t) * TILE_BYTES, &maps.x[t], &full[s], k, brow);
          tma_load_2d(st + (TERMS + 2 * t + 1) * TILE_BYTES, &maps.z[t], &full[s], k, brow);
        }
        issued = kb + 1;
      }
      // after an abort, every load already issued must land before the CTA may exit
      if (*abort_flag) {
        for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
          mbar_wait_timer(&full[kb % STAGES], (kb / STAGES) & 1);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      // N = 256: the B operand is X (rows 0-127, giving Re) stacked on Z
      // (rows 128-255, giving Im), so one MMA fills both accumulators
      constexpr uint32_t idesc = idesc_bf16(BM, 2 * BN);
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        if (!mbar_wait(&full[s], (kb / STAGES) & 1, abort_flag)) {
          *abort_flag = 1;
          atomicExch(err, 2);
          break;
        }
        const int f = kb / fold;
        const int b = f & 1;
        const bool first = (kb % fold) == 0;
        if (first && f >= 2 && !mbar_wait(&tempty[b], ((f >> 1) - 1) & 1, abort_flag)) {
          *abort_flag = 1;
          atomicExch(err, 3);
          break;
        }
        tc_fence_after();
        const uint32_t st = smem_u32(smem + s * C::STAGE_BYTES);
        const uint32_t d = tmem + b * 256;  // Re in columns 0-127, Im in 128-255
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint32_t koff = kk * 32;  // 16 bf16 = 32 bytes along K inside the swizzle atom
          uint64_t da[3], db[3];
#pragma unroll
          for (int t = 0; t < TERMS; ++t) {
            da[t] = kmajor_desc<BK>(st + t * TILE_BYTES + koff);
            db[t] = kmajor_desc<BK>(st + (TERMS + 2 * t) * TILE_BYTES + koff);
          }
          const uint32_t acc = (first && kk == 0) ? 0u : 1u;
          // hi*hi, hi*lo, lo*hi  (three terms: + hi*mid, mid*hi, mid*mid, hi*lo, lo*hi)
          umma(d, da[0], db[0], idesc, acc);
          umma(d, da[0], db[1], idesc, 1u);
          umma(d, da[1], db[0], idesc, 1u);
          if (TERMS == 3) {
            umma(d, da[1], db[1], idesc, 1u);
            umma(d, da[0], db[2], idesc, 1u);
            umma(d, da[2], db[0], idesc, 1u);
          }
        }
        umma_commit(&empty[s]);
        if ((kb % fold) == fold - 1 || kb == nk - 1) umma_commit(&tfull[b]);
      }
      // every MMA issued so far must finish before TMEM is released
      umma_commit(mma_done);
      if (!mbar_wait_timer(mma_done, 0)) atomicExch(err, 5);
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 2..17)
    // Warp w reads TMEM lane quarter w % 4 (rows 32q..32q+31) and column
    // slice cs = (w - 2) / 4 (32 columns) of the Re and Im accumulators; four
    // warps per quarter drain a fold in a quarter of the time one would.  The
    // FP32 partial of every fold is added to FP32 running sums held in
    // registers (round to nearest) and the running sums go to the FP64 chi0
    // every `flush` folds, so the truncating accumulation inside the tensor
    // core never spans more than one fold.
    const int q = warp & 3;
    const int cs = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    const int gi = i0 + row;
    const int cbase = cs * 32;
    double2* crow = GEMM ? nullptr : chi + ((int64_t)w * NG + gi) * NG + j0 + cbase;
    // HERK: columns of this thread in the lower triangle and the sphere;
    // GEMM: columns inside the sphere of a row inside the pair range
    int ncol;
    if constexpr (GEMM)
      ncol = (gi < ga.P) ? max(0, min(32, NG - (j0 + cbase))) : 0;
    else
      ncol = (gi < NG) ? max(0, min(32, min(NG, gi + 1) - (j0 + cbase))) : 0;
    float wrow = 0.f;  // GEMM: 2 wgt[w][p] of the current frequency
    int wcur = -1;
    float sre[32], sim[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) sre[c] = sim[c] = 0.f;
#define RPA_TC_FLUSH()                                      \
  do {                                                      \
    _Pragma("unroll") for (int c = 0; c < 32; ++c) {        \
      if (c < ncol) {                                       \
        double2 v = crow[c];                                \
        v.x += (double)sre[c];                              \
        v.y += (double)sim[c];                              \
        crow[c] = v;                                        \
      }                                                     \
      sre[c] = 0.f;                                         \
      sim[c] = 0.f;                                         \
    }                                                       \
  } while (0)
    if constexpr (GEMM) flush = 1 << 30;  // one write at the end
    for (int f = 0; f < nfold; ++f) {
      const int b = f & 1;
      // the warp decides together: tcgen05.ld below is warp-collective
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&tfull[b], (f >> 1) & 1, abort_flag));
      if (!ok) {
        *abort_flag = 1;
        atomicExch(err, 4);
        break;
      }
      tc_fence_after();
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + b * 256 + cbase;
      float sc = 1.f;
      if constexpr (GEMM) {
        const int wf = (f * fold) / ga.nkw;  // folds never straddle frequencies (fold divides nkw)
        if (wf != wcur) {
          wcur = wf;
          wrow = gi >= ga.P ? 0.f : ga.wgt ? 2.f * ga.wgt[(int64_t)wf * ga.P + gi] : 1.f;
        }
        sc = wrow;
      }
      // 18 warps leave 96 registers a thread: 64 running sums and one
      // 16-column load at a time; the buffer is released as soon as the last
      // load has landed, before its additions
      float v[16];
      tmem_ld16(base, v);
#pragma unroll
      for (int c = 0; c < 16; ++c) sre[c] = fmaf(sc, v[c], sre[c]);
      tmem_ld16(base + 16, v);
#pragma unroll
      for (int c = 0; c < 16; ++c) sre[16 + c] = fmaf(sc, v[c], sre[16 + c]);
      tmem_ld16(base + 128, v);
#pragma unroll
      for (int c = 0; c < 16; ++c) sim[c] = fmaf(sc, v[c], sim[c]);
      tmem_ld16(base + 144, v);
      tc_fence_before();
      mbar_arrive(&tempty[b]);
#pragma unroll
      for (int c = 0; c < 16; ++c) sim[16 + c] = fmaf(sc, v[c], sim[16 + c]);
      if ((f + 1) % flush == 0) RPA_TC_FLUSH();
    }
    if constexpr (GEMM) {
      float2* orow = ga.out + (int64_t)w * ga.out_batch + (int64_t)gi * NG + j0 + cbase;
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c < ncol) {
          float2 o = make_float2(sre[c], sim[c]);
          if (ga.accumulate) {
            const float2 v = orow[c];
            o.x += v.x;
            o.y += v.y;
          }
          orow[c] = o;
        }
    } else {
      RPA_TC_FLUSH();
    }
#undef RPA_TC_FLUSH
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ---------------------------------------------------------------- operand preparation
__device__ __forceinline__ void split2(float x, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  l = __float2bfloat16_rn(x - __bfloat162float(h));
}
__device__ __forceinline__ void split3(float x, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// X[t][g][2p+c], Z[t][g][2p+c] from N[p][g] (transpose through shared memory), zero padding.
template <int TERMS>
__global__ void __launch_bounds__(256) prep_xz_kernel(const float2* __restrict__ N, int64_t P, int NG, int NGpad,
                                                      int64_t Kpad, __nv_bfloat162* __restrict__ X,
                                                      __nv_bfloat162* __restrict__ Z, int64_t term_stride) {
  __shared__ float2 t[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int64_t p0 = (int64_t)blockIdx.y * 32;
  const int g0 = blockIdx.x * 32;
  for (int r = ty; r < 32; r += 8) {
    const int64_t p = p0 + r;
    const int g = g0 + tx;
    t[r][tx] = (p < P && g < NG) ? N[p * NG + g] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int g = g0 + r;
    const int64_t p = p0 + tx;
    const float2 v = t[tx][r];
    const int64_t o = (int64_t)g * (Kpad / 2) + p;
    __nv_bfloat16 rh, rm, rl, ih, im, il;
    if (TERMS == 2) {
      split2(v.x, rh, rl);
      split2(v.y, ih, il);
      X[o] = __halves2bfloat162(rh, ih);
      X[o + term_stride] = __halves2bfloat162(rl, il);
      Z[o] = __halves2bfloat162(__hneg(ih), rh);
      Z[o + term_stride] = __halves2bfloat162(__hneg(il), rl);
    } else {
      split3(v.x, rh, rm, rl);
      split3(v.y, ih, im, il);
      X[o] = __halves2bfloat162(rh, ih);
      X[o + term_stride] = __halves2bfloat162(rm, im);
      X[o + 2 * term_stride] = __halves2bfloat162(rl, il);
      Z[o] = __halves2bfloat162(__hneg(ih), rh);
      Z[o + term_stride] = __halves2bfloat162(__hneg(im), rm);
      Z[o + 2 * term_stride] = __halves2bfloat162(__hneg(il), rl);
    }
  }
}

// A[t][w][g][2p+c] = split(w_p(w) * (Re, Im) N[p][g]) for every frequency.
template <int TERMS>
__global__ void __launch_bounds__(256) prep_a_kernel(const float2* __restrict__ N, const float* __restrict__ wgt,
                                                     int64_t P, int NG, int NGpad, int64_t Kpad, int nw,
                                                     __nv_bfloat162* __restrict__ A, int64_t term_stride) {
  __shared__ float2 t[32][33];
  __shared__ float ws[32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t p0 = (int64_t)blockIdx.y * 32;
  const int g0 = blockIdx.x * 32;
  for (int r = ty; r < 32; r += 8) {
    const int64_t p = p0 + r;
    const int g = g0 + tx;
    t[r][tx] = (p < P && g < NG) ? N[p * NG + g] : make_float2(0.f, 0.f);
  }
  for (int w = 0; w < nw; ++w) {
    __syncthreads();
    if (threadIdx.x < 32) {
      const int64_t p = p0 + threadIdx.x;
      ws[threadIdx.x] = p < P ? wgt[(int64_t)w * P + p] : 0.f;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int g = g0 + r;
      const float2 v = t[tx][r];
      const float wp = ws[tx];
      const int64_t o = ((int64_t)w * NGpad + g) * (Kpad / 2) + p0 + tx;
      __nv_bfloat16 rh, rm, rl, ih, im, il;
      if (TERMS == 2) {
        split2(wp * v.x, rh, rl);
        split2(wp * v.y, ih, il);
        A[o] = __halves2bfloat162(rh, ih);
        A[o + term_stride] = __halves2bfloat162(rl, il);
      } else {
        split3(wp * v.x, rh, rm, rl);
        split3(wp * v.y, ih, im, il);
        A[o] = __halves2bfloat162(rh, ih);
        A[o + term_stride] = __halves2bfloat162(rm, im);
        A[o + 2 * term_stride] = __halves2bfloat162(rl, il);
      }
    }
  }
}

// B operand of the PAW product from R[y][kp][g] (one batch y per occupied
// band): with b = conj R, X[t][y NGpad + g][2 kp + c] = split(Re b, Im b) and
// Z = split(-Im b, Re b); rows to NGpad and K to KN = 2 * round32(KP), zero
// padding (transpose through shared memory).
template <int TERMS>
__global__ void __launch_bounds__(256) prep_r_kernel(const float2* __restrict__ R, int KP, int NG, int NGpad,
                                                     int64_t KN, __nv_bfloat162* __restrict__ X,
                                                     __nv_bfloat162* __restrict__ Z, int64_t term_stride) {
  __shared__ float2 t[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int y = blockIdx.z;
  const float2* Ry = R + (int64_t)y * KP * NG;
  const int k0 = blockIdx.y * 32, g0 = blockIdx.x * 32;
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r, g = g0 + tx;
    t[r][tx] = (k < KP && g < NG) ? Ry[(int64_t)k * NG + g] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int g = g0 + r;
    const float2 v = t[tx][r];
    const int64_t o = ((int64_t)y * NGpad + g) * (KN / 2) + k0 + tx;
    // b = (v.x, -v.y): X = (v.x, -v.y), Z = (v.y, v.x); the split is odd in its argument
    __nv_bfloat16 rh, rm, rl, ih, im, il;
    if (TERMS == 2) {
      split2(v.x, rh, rl);
      split2(v.y, ih, il);
      X[o] = __halves2bfloat162(rh, __hneg(ih));
      X[o + term_stride] = __halves2bfloat162(rl, __hneg(il));
      Z[o] = __halves2bfloat162(ih, rh);
      Z[o + term_stride] = __halves2bfloat162(il, rl);
    } else {
      split3(v.x, rh, rm, rl);
      split3(v.y, ih, im, il);
      X[o] = __halves2bfloat162(rh, __hneg(ih));
      X[o + term_stride] = __halves2bfloat162(rm, __hneg(im));
      X[o + 2 * term_stride] = __halves2bfloat162(rl, __hneg(il));
      Z[o] = __halves2bfloat162(ih, rh);
      Z[o + term_stride] = __halves2bfloat162(im, rm);
      Z[o + 2 * term_stride] = __halves2bfloat162(il, rl);
    }
  }
}

// A[t][p][2k+c] = split((Re, Im) N[p][k]) for the adjoint product: rows padded
// to Prows, K to KN = 2 * round32(NG), zero padding.
template <int TERMS>
__global__ void __launch_bounds__(256) prep_n_kernel(const float2* __restrict__ N, int64_t P, int NG, int64_t Prows,
                                                     int KN, __nv_bfloat162* __restrict__ A, int64_t term_stride) {
  const int kh = KN / 2;
  const int64_t total = Prows * kh;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(id % kh);
    const int64_t p = id / kh;
    const float2 v = (p < P && k < NG) ? N[p * NG + k] : make_float2(0.f, 0.f);
    __nv_bfloat16 rh, rm, rl, ih, im, il;
    if (TERMS == 2) {
      split2(v.x, rh, rl);
      split2(v.y, ih, il);
      A[id] = __halves2bfloat162(rh, ih);
      A[id + term_stride] = __halves2bfloat162(rl, il);
    } else {
      split3(v.x, rh, rm, rl);
      split3(v.y, ih, im, il);
      A[id] = __halves2bfloat162(rh, ih);
      A[id + term_stride] = __halves2bfloat162(rm, im);
      A[id + 2 * term_stride] = __halves2bfloat162(rl, il);
    }
  }
}

// ---------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

static bool make_map(CUtensorMap* m, const void* base, int64_t K, int64_t rows, int bk) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(K * 2)};
  cuuint32_t box[2] = {(cuuint32_t)bk, BM};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

struct Geometry {
  int NGpad;
  int64_t Ppad, Kpad;
};
static Geometry geometry(int64_t P, int NG) {
  Geometry g;
  g.NGpad = (NG + BM - 1) / BM * BM;
  g.Ppad = (P + 31) / 32 * 32;
  g.Kpad = 2 * g.Ppad;
  return g;
}

}  // namespace tc

size_t herk_tc_scratch_bytes(int64_t P, int NG, int nw, int terms) {
  const tc::Geometry g = tc::geometry(P, NG);
  const size_t op = (size_t)g.NGpad * g.Kpad * 2;  // one bf16 operand matrix
  return op * (size_t)terms * (size_t)(nw + 2);
}

template <int TERMS, int BK, int STAGES>
static cudaError_t launch_gemm(const tc::Maps& maps, dim3 grid, int NG, int NGpad, int64_t Kpad, int fold64, int flush,
                               double2* chi, int* err, cudaStream_t s) {
  using namespace tc;
  using C = Cfg<TERMS, BK, STAGES>;
  static_assert(C::SMEM_BYTES <= 227 * 1024, "shared-memory ring too large");
  const int nk = (int)(Kpad / BK);
  // the fold length counts 64-element units of three products (two terms);
  // with three terms (six products per element) a unit is 32 elements, so a
  // fold holds the same number of truncating tensor-core accumulations
  const int fold = TERMS == 3 ? fold64 * (32 / BK) : fold64 * (64 / BK);
  cudaError_t e = cudaFuncSetAttribute(herk_tc_kernel<TERMS, BK, STAGES, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  herk_tc_kernel<TERMS, BK, STAGES, false><<<grid, NUM_THREADS, C::SMEM_BYTES, s>>>(maps, NG, NGpad, nk, fold, flush,
                                                                                   chi, err, GemmArgs{});
  return cudaGetLastError();
}

// Bounds shared by the two calls below.
static cudaError_t check_args(int64_t P, int NG, int nw, int terms, size_t scratch_bytes) {
  if (terms != 2 && terms != 3) return cudaErrorInvalidValue;
  const tc::Geometry g = tc::geometry(P, NG);
  if (scratch_bytes < herk_tc_scratch_bytes(P, NG, nw, terms)) return cudaErrorInvalidValue;
  if (g.Kpad > (int64_t)1 << 31 || (int64_t)nw * g.NGpad > (1 << 30)) return cudaErrorInvalidValue;
  return cudaSuccess;
}

// Scratch layout: X terms, Z terms, then the per-frequency A terms.
struct Operands {
  __nv_bfloat16 *X, *Z, *A;
  int64_t op_elems;
};
static Operands operands(void* scratch, const tc::Geometry& g, int terms) {
  Operands o;
  o.op_elems = (int64_t)g.NGpad * g.Kpad;
  o.X = (__nv_bfloat16*)scratch;
  o.Z = o.X + o.op_elems * terms;
  o.A = o.Z + o.op_elems * terms;
  return o;
}

cudaError_t herk_tc_prepare(const float2* N, int64_t P, int NG, const float* wgt, int nw, int terms, void* scratch,
                            size_t scratch_bytes, cudaStream_t s) {
  using namespace tc;
  if (P == 0 || NG == 0 || nw == 0) return cudaSuccess;
  cudaError_t e = check_args(P, NG, nw, terms, scratch_bytes);
  if (e != cudaSuccess) return e;
  const Geometry g = geometry(P, NG);
  const Operands o = operands(scratch, g, terms);
  dim3 pg(g.NGpad / 32, (unsigned)(g.Ppad / 32));
  if (terms == 3) {
    prep_xz_kernel<3><<<pg, 256, 0, s>>>(N, P, NG, g.NGpad, g.Kpad, (__nv_bfloat162*)o.X, (__nv_bfloat162*)o.Z,
                                         o.op_elems / 2);
    prep_a_kernel<3><<<pg, 256, 0, s>>>(N, wgt, P, NG, g.NGpad, g.Kpad, nw, (__nv_bfloat162*)o.A,
                                        o.op_elems * nw / 2);
  } else {
    prep_xz_kernel<2><<<pg, 256, 0, s>>>(N, P, NG, g.NGpad, g.Kpad, (__nv_bfloat162*)o.X, (__nv_bfloat162*)o.Z,
                                         o.op_elems / 2);
    prep_a_kernel<2><<<pg, 256, 0, s>>>(N, wgt, P, NG, g.NGpad, g.Kpad, nw, (__nv_bfloat162*)o.A,
                                        o.op_elems * nw / 2);
  }
  return cudaGetLastError();
}

cudaError_t herk_tc_run(int64_t P, int NG, int nw, int terms, int fold_stages, int flush_folds, int pipe,
                        double2* chi, void* scratch, size_t scratch_bytes, int* err, cudaStream_t s) {
  using namespace tc;
  if (P == 0 || NG == 0 || nw == 0) return cudaSuccess;
  cudaError_t e = check_args(P, NG, nw, terms, scratch_bytes);
  if (e != cudaSuccess) return e;
  if (fold_stages < 1) fold_stages = 1;
  if (flush_folds < 1) flush_folds = 1;
  // three terms: 9 tiles a stage, so 32-element stages x 3 (217 KB); two
  // terms: 64-element stages x 2 (default) or 32-element stages x 4
  const int bk = (terms == 3 || pipe == 1) ? 32 : 64;
  const Geometry g = geometry(P, NG);
  const Operands o = operands(scratch, g, terms);
  Maps maps;
  memset(&maps, 0, sizeof(maps));
  for (int t = 0; t < terms; ++t) {
    if (!make_map(&maps.a[t], o.A + o.op_elems * nw * t, g.Kpad, (int64_t)nw * g.NGpad, bk) ||
        !make_map(&maps.x[t], o.X + o.op_elems * t, g.Kpad, g.NGpad, bk) ||
        !make_map(&maps.z[t], o.Z + o.op_elems * t, g.Kpad, g.NGpad, bk))
      return cudaErrorInvalidValue;
  }
  const int nt = g.NGpad / BM;
  dim3 grid(nt * (nt + 1) / 2, nw);
  if (terms == 3)
    return launch_gemm<3, 32, 3>(maps, grid, NG, g.NGpad, g.Kpad, fold_stages, flush_folds, chi, err, s);
  if (bk == 32) return launch_gemm<2, 32, 4>(maps, grid, NG, g.NGpad, g.Kpad, fold_stages, flush_folds, chi, err, s);
  return launch_gemm<2, 64, 2>(maps, grid, NG, g.NGpad, g.Kpad, fold_stages, flush_folds, chi, err, s);
}

// ---------------------------------------------------------------- adjoint product on the tensor cores
// out[p][g] = 2 sum_w wgt[w][p] sum_k N[p][k] conj(Gam_w[k][g]) for Hermitian
// Gam_w (the adjoint of the rank-k update).  Gam is split once per q-point into
// X / Z operands [terms][nw * NGpad][KN]; the pair densities of each block into
// A [terms][Prows][KN].
static int64_t nbar_kn(int NG) { return 2 * (((int64_t)NG + 31) / 32 * 32); }
static int64_t nbar_prows(int64_t P) { return (P + tc::BM - 1) / tc::BM * tc::BM; }

size_t nbar_tc_gam_bytes(int NG, int nw, int terms) {
  const int64_t NGpad = (NG + tc::BM - 1) / tc::BM * tc::BM;
  return (size_t)2 * terms * nw * NGpad * nbar_kn(NG) * 2;
}
size_t nbar_tc_a_bytes(int64_t P, int NG, int terms) { return (size_t)terms * nbar_prows(P) * nbar_kn(NG) * 2; }

cudaError_t nbar_tc_prepare_gam(const float2* Gam, int NG, int nw, int terms, void* gbuf, cudaStream_t s) {
  if (terms != 2 && terms != 3) return cudaErrorInvalidValue;
  const int NGpad = (NG + tc::BM - 1) / tc::BM * tc::BM;
  const int64_t KN = nbar_kn(NG);
  const int64_t op = (int64_t)nw * NGpad * KN / 2;  // bf16 pairs per term of X (or Z)
  __nv_bfloat162* X = (__nv_bfloat162*)gbuf;
  __nv_bfloat162* Z = X + op * terms;
  dim3 pg(NGpad / 32, (unsigned)(KN / 2 / 32));
  for (int w = 0; w < nw; ++w) {
    const float2* Gw = Gam + (int64_t)w * NG * NG;
    const int64_t off = (int64_t)w * NGpad * KN / 2;
    // rows k of Gam play the role of pairs: X[g][2k] = (Re, Im) Gam[k][g], Z = (-Im, Re)
    if (terms == 3)
      tc::prep_xz_kernel<3><<<pg, 256, 0, s>>>(Gw, NG, NG, NGpad, KN, X + off, Z + off, op);
    else
      tc::prep_xz_kernel<2><<<pg, 256, 0, s>>>(Gw, NG, NG, NGpad, KN, X + off, Z + off, op);
  }
  return cudaGetLastError();
}

cudaError_t nbar_tc_run(const float2* N, const float* wgt, int64_t P, int NG, int nw, int terms, const void* gbuf,
                        void* abuf, size_t abytes, float2* out, int* err, cudaStream_t s) {
  using namespace tc;
  if (P == 0 || NG == 0 || nw == 0) return cudaSuccess;
  if ((terms != 2 && terms != 3) || abytes < nbar_tc_a_bytes(P, NG, terms)) return cudaErrorInvalidValue;
  const int NGpad = (NG + BM - 1) / BM * BM;
  const int64_t KN = nbar_kn(NG), Prows = nbar_prows(P);
  if (Prows > (1 << 30) || (int64_t)nw * NGpad > (1 << 30)) return cudaErrorInvalidValue;
  const int64_t aterm = Prows * KN / 2;
  {
    const int64_t total = Prows * KN / 2;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 32);
    if (terms == 3)
      prep_n_kernel<3><<<blocks, 256, 0, s>>>(N, P, NG, Prows, (int)KN, (__nv_bfloat162*)abuf, aterm);
    else
      prep_n_kernel<2><<<blocks, 256, 0, s>>>(N, P, NG, Prows, (int)KN, (__nv_bfloat162*)abuf, aterm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int bk = terms == 3 ? 32 : 64;
  const int64_t gop = (int64_t)nw * NGpad * KN;  // bf16 elements per term of X
  const __nv_bfloat16* X = (const __nv_bfloat16*)gbuf;
  const __nv_bfloat16* Z = X + gop * terms;
  const __nv_bfloat16* A = (const __nv_bfloat16*)abuf;
  Maps maps;
  memset(&maps, 0, sizeof(maps));
  for (int t = 0; t < terms; ++t) {
    if (!make_map(&maps.a[t], A + Prows * KN * t, KN, Prows, bk) ||
        !make_map(&maps.x[t], X + gop * t, KN, (int64_t)nw * NGpad, bk) ||
        !make_map(&maps.z[t], Z + gop * t, KN, (int64_t)nw * NGpad, bk))
      return cudaErrorInvalidValue;
  }
  GemmArgs ga;
  ga.P = P;
  ga.nkw = (int)(KN / bk);
  ga.ngt = NGpad / BN;
  ga.wgt = wgt;
  ga.out = out;
  ga.nwb = nw;
  ga.accumulate = 0;
  ga.out_batch = 0;
  const int nk = ga.nkw * nw;
  const dim3 grid((unsigned)((Prows / BM) * ga.ngt), 1);
  cudaError_t e;
  if (terms == 3) {
    using C = Cfg<3, 32, 3>;
    if ((e = cudaFuncSetAttribute(herk_tc_kernel<3, 32, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  C::SMEM_BYTES)) != cudaSuccess)
      return e;
    herk_tc_kernel<3, 32, 3, true><<<grid, NUM_THREADS, C::SMEM_BYTES, s>>>(maps, NG, NGpad, nk, 1, 1, nullptr, err,
                                                                           ga);
  } else {
    using C = Cfg<2, 64, 2>;
    if ((e = cudaFuncSetAttribute(herk_tc_kernel<2, 64, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  C::SMEM_BYTES)) != cudaSuccess)
      return e;
    herk_tc_kernel<2, 64, 2, true><<<grid, NUM_THREADS, C::SMEM_BYTES, s>>>(maps, NG, NGpad, nk, 1, 1, nullptr, err,
                                                                           ga);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- PAW term on the tensor cores
// N[(y nR + b)][g] += sum_kp Pm[b][kp] R[y][kp][g] (Eq. 6 with the factor R of
// each occupied band y) as the unweighted batched variant of the kernel: A =
// split Pm [terms][Prows][KN], B = split conj R [terms][nL NGpad][KN] as X / Z.
size_t paw_tc_bytes(int nL, int nR, int KP, int NG, int terms) {
  const int64_t NGpad = (NG + tc::BM - 1) / tc::BM * tc::BM;
  const int64_t KN = nbar_kn(KP);
  return (size_t)terms * ((size_t)nbar_prows(nR) * KN + (size_t)2 * nL * NGpad * KN) * 2;
}

cudaError_t paw_tc_run(const float2* Pm, const float2* R, int KP, int nL, int nR, int NG, int terms, void* scratch,
                       size_t bytes, float2* N, int* err, cudaStream_t s) {
  using namespace tc;
  if (nL == 0 || nR == 0 || NG == 0 || KP == 0) return cudaSuccess;
  if ((terms != 2 && terms != 3) || bytes < paw_tc_bytes(nL, nR, KP, NG, terms)) return cudaErrorInvalidValue;
  const int NGpad = (NG + BM - 1) / BM * BM;
  const int64_t KN = nbar_kn(KP), Prows = nbar_prows(nR);
  if ((int64_t)nL * NGpad > (1 << 30) || nL > 65535) return cudaErrorInvalidValue;
  const int64_t aop = Prows * KN, bop = (int64_t)nL * NGpad * KN;  // bf16 elements per term
  __nv_bfloat16* A = (__nv_bfloat16*)scratch;
  __nv_bfloat16* X = A + aop * terms;
  __nv_bfloat16* Z = X + bop * terms;
  {
    const int64_t total = Prows * KN / 2;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 32);
    const dim3 pg(NGpad / 32, (unsigned)(KN / 2 / 32), nL);
    if (terms == 3) {
      prep_n_kernel<3><<<blocks, 256, 0, s>>>(Pm, nR, KP, Prows, (int)KN, (__nv_bfloat162*)A, aop / 2);
      prep_r_kernel<3><<<pg, 256, 0, s>>>(R, KP, NG, NGpad, KN, (__nv_bfloat162*)X, (__nv_bfloat162*)Z, bop / 2);
    } else {
      prep_n_kernel<2><<<blocks, 256, 0, s>>>(Pm, nR, KP, Prows, (int)KN, (__nv_bfloat162*)A, aop / 2);
      prep_r_kernel<2><<<pg, 256, 0, s>>>(R, KP, NG, NGpad, KN, (__nv_bfloat162*)X, (__nv_bfloat162*)Z, bop / 2);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int bk = terms == 3 ? 32 : 64;
  Maps maps;
  memset(&maps, 0, sizeof(maps));
  for (int t = 0; t < terms; ++t) {
    if (!make_map(&maps.a[t], A + aop * t, KN, Prows, bk) ||
        !make_map(&maps.x[t], X + bop * t, KN, (int64_t)nL * NGpad, bk) ||
        !make_map(&maps.z[t], Z + bop * t, KN, (int64_t)nL * NGpad, bk))
      return cudaErrorInvalidValue;
  }
  GemmArgs ga;
  ga.P = nR;
  ga.nkw = (int)(KN / bk);
  ga.ngt = NGpad / BN;
  ga.wgt = nullptr;
  ga.out = N;
  ga.nwb = 1;
  ga.accumulate = 1;
  ga.out_batch = (int64_t)nR * NG;
  const int nk = ga.nkw;
  const dim3 grid((unsigned)((Prows / BM) * ga.ngt), (unsigned)nL);
  cudaError_t e;
  if (terms == 3) {
    using C = Cfg<3, 32, 3>;
    if ((e = cudaFuncSetAttribute(herk_tc_kernel<3, 32, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  C::SMEM_BYTES)) != cudaSuccess)
      return e;
    herk_tc_kernel<3, 32, 3, true><<<grid, NUM_THREADS, C::SMEM_BYTES, s>>>(maps, NG, NGpad, nk, 1, 1, nullptr, err,
                                                                           ga);
  } else {
    using C = Cfg<2, 64, 2>;
    if ((e = cudaFuncSetAttribute(herk_tc_kernel<2, 64, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  C::SMEM_BYTES)) != cudaSuccess)
      return e;
    herk_tc_kernel<2, 64, 2, true><<<grid, NUM_THREADS, C::SMEM_BYTES, s>>>(maps, NG, NGpad, nk, 1, 1, nullptr, err,
                                                                           ga);
  }
  return cudaGetLastError();
}

}  // namespace rpa
