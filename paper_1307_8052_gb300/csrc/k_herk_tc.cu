// Tensor-core grouped Hermitian rank-k update of chi0 (Eq. 17, the paper's
// "multi-u" zherk) for every frequency, on the 5th-generation tensor cores.
//
// Real-stacked form.  With a_p = n_p(G_i), b_p = n_p(G_j) and the K index
// k = 2p + c running over (pair, re/im):
//   Re chi_ij = sum_k A_ik X_jk,  Im chi_ij = sum_k A_ik Z_jk,
//   A = w_p(w) (Re a, Im a),  X = (Re b, Im b),  Z = (-Im b, Re b).
// The weight w_p(w) of Eq. 16 multiplies along K (one pair per two K
// elements), so it is applied to the A operand before the product.
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
// splits (K-major, bfloat16) and, for two terms, one FP32 copy F of the pair
// densities in the same K order (frequency independent).  The kernel streams
// 128-row tiles with TMA (cp.async.bulk.tensor; 64-element stages with the
// 128-byte swizzle in a 2-stage ring, or 32-element stages with the 64-byte
// swizzle for three terms).  With two terms the A slots of a stage receive the
// FP32 rows of F, and two converter warps scale every pair by w_p(w) of the
// CTA's frequency and split it into the bfloat16 hi and lo tiles in place
// (fused weighting: no per-frequency operand is stored).  With three terms, or
// when the fused form is switched off, a second prep kernel writes the
// weighted A splits of every frequency instead.  One thread issues one
// tcgen05.mma (M = 128, N = 256, K = 16) per product with the X tile stacked on
// the Z tile, so Re and Im land in one 256-column TMEM buffer; two such buffers
// alternate, and sixteen epilogue warps drain one with tcgen05.ld while the
// MMAs fill the other (warps whose rows are padding or whose columns lie above
// the diagonal skip the loads).  Only lower-triangle tiles are launched.  A
// batched product variant (GEMM = true) serves the adjoint and the PAW term.
// Every wait is bounded by the GPU global timer (a runtime limit); on timeout
// the CTA raises a flag, waits for the loads and products it issued, frees
// TMEM and exits.
#include "rpa_internal.h"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

namespace rpa {
namespace tc {

constexpr int BM = 128;               // tile rows (G_i)
constexpr int BN = 128;               // tile cols (G_j)
constexpr int EPI_WARPS = 16;         // epilogue warps: 4 per TMEM lane quarter
constexpr int CONV_WARPS = 2;         // converter warps of the fused weighting
constexpr int EPI_WARP0 = 2 + CONV_WARPS;  // first epilogue warp (a multiple of 4: warp % 4 is its lane quarter)
// warp 0 TMA, warp 1 MMA, warps 2-3 converters, warps 4-19 epilogue
constexpr int NUM_THREADS = 32 * (EPI_WARP0 + EPI_WARPS);
// limit of the waits for work a CTA has already issued (loads landing,
// products finishing) before it frees tensor memory and exits
constexpr uint64_t DRAIN_NS = 4000000000ull;

// Pipeline shapes: BK bf16 K-elements per stage (64: 128-byte rows with the
// 128-byte swizzle; 32: 64-byte rows with the 64-byte swizzle) and STAGES
// stages in the shared-memory ring.
// Unfused: one ring of STAGES stages, each the A terms then the B tiles.
// Fused (two terms): a ring of STAGES B stages, then a ring of AST = 3 A stages
// (the FP32 rows of F, converted in place), so the A rows of a stage are
// loaded and converted two MMA stages ahead of their use (224 KB).
template <int TERMS, int BK_, int STAGES_, bool FUSED = false> struct Cfg {
  static constexpr int BK = BK_;
  static constexpr int STAGES = STAGES_;
  static constexpr int AST = FUSED ? 3 : STAGES_;   // A-ring depth
  static constexpr int TILE_BYTES = BM * BK * 2;
  static constexpr int A_TILES = TERMS;             // A hi, (mid), lo
  static constexpr int B_TILES = 2 * TERMS;         // per term X then Z: one 256-row B operand
  static constexpr int A_BYTES = A_TILES * TILE_BYTES;
  static constexpr int B_BYTES = B_TILES * TILE_BYTES;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int RING_BYTES = FUSED ? STAGES * B_BYTES + AST * A_BYTES : STAGES * STAGE_BYTES;
  static constexpr int SMEM_BYTES = RING_BYTES + 1024 + 256;
  static_assert(STAGES <= 4 && AST <= 4, "barrier area holds up to 4 stages per ring");
  __device__ static unsigned char* a_ptr(unsigned char* smem, int s) {
    return FUSED ? smem + STAGES * B_BYTES + s * A_BYTES : smem + s * STAGE_BYTES;
  }
  __device__ static unsigned char* b_ptr(unsigned char* smem, int s) {
    return FUSED ? smem + s * B_BYTES : smem + s * STAGE_BYTES + A_BYTES;
  }
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
// Bounded wait: false if the limit expired or another role aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (gtimer() - t0 > limit_ns) return false;
  }
}

// Warp-collective bounded wait: lane 0 spins, the result is broadcast, and
// every lane then observes the completed phase itself (it cannot move on: its
// next phase needs this warp's own arrival), so each lane acquires what the
// phase released.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          uint64_t limit_ns) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort_flag, limit_ns) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  return __all_sync(0xffffffffu, ok && mbar_try_wait(bar, parity));
}

// Bounded wait for work already issued (abort path), ignoring the abort flag.
__device__ __forceinline__ bool mbar_wait_timer(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = gtimer();
  while (!mbar_try_wait(bar, parity))
    if (gtimer() - t0 > DRAIN_NS) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int k, int row) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(k), "r"(row)
      : "memory");
}

// Multicast form: the tile lands at the same shared-memory offset in every CTA
// of ctaMask and completes bytes on the mbarrier at the same offset in each.
__device__ __forceinline__ void tma_load_2d_mc(void* dst, const CUtensorMap* map, uint64_t* bar, int k, int row,
                                               uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1, {%3, "
      "%4}], [%2], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(k), "r"(row), "h"(mask)
      : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// all threads of every CTA of the cluster
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
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
// arrive once on the mbarrier at this offset in every CTA of ctaMask when the
// issued products are done
__device__ __forceinline__ void umma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                   smem_u32(bar)),
               "h"(mask)
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
  CUtensorMap a[3];  // weighted A terms (rows = w * NGpad + i); fused: a[0] = FP32 F (rows i)
  CUtensorMap x[3];  // X terms
  CUtensorMap z[3];  // Z terms
};

// Run-time controls of the kernel.
struct Ctl {
  uint64_t wait_ns;    // limit of every wait on another role's progress
  int stall_stage;     // >= 0: the producer withholds this K stage and all later ones (test of the timeout path)
  const float* wpad;   // fused weighting: weights [nw][wstride], zero past the last pair
  int64_t wstride;
};

// The FP32 source F of the fused weighting stores each 64-element K block of a
// row as two 32-float halves: 16-byte chunk c of half h holds the K elements
// 8c + 4h + (0..3).  A stage loads the two halves into the A hi and A lo tile
// slots (128-byte rows, 128-byte swizzle); chunk c of both halves holds exactly
// the four pairs whose hi and lo bfloat16 values form chunk c of the A hi and
// A lo tiles, so every chunk converts in place.
__host__ __device__ constexpr int64_t f_pos(int64_t k) {
  return (k & ~(int64_t)63) + ((k >> 2) & 1) * 32 + ((k & 63) >> 3) * 4 + (k & 3);
}

// (x, y) -> bfloat16 hi = rn(x, y) and lo = rn((x, y) - hi), packed low = x.
__device__ __forceinline__ void split_pair(float x, float y, uint32_t& h, uint32_t& l) {
  const __nv_bfloat162 hb = __floats2bfloat162_rn(x, y);
  const float2 hf = __bfloat1622float2(hb);
  const __nv_bfloat162 lb = __floats2bfloat162_rn(__fsub_rn(x, hf.x), __fsub_rn(y, hf.y));
  h = *reinterpret_cast<const uint32_t*>(&hb);
  l = *reinterpret_cast<const uint32_t*>(&lb);
}

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

// CL = 2: the CTAs of a cluster pair are the same tile at frequencies 2c and
// 2c + 1, whose B operand (X, Z: unweighted) is the same.  Each loads every
// other B tile of a stage for both (TMA multicast), so a CTA fetches its A
// tiles and half of B; a stage slot is reused once the products of both CTAs
// have read it (each MMA commit arrives on the slot's barrier in both CTAs).
// Same loads, products and order as CL = 1: chi0 is bit-identical.
template <int TERMS, int BK, int STAGES, bool GEMM, bool FUSED, int CL>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    herk_tc_kernel(const __grid_constant__ Maps maps, int NG, int NGpad, int nk, int fold, int flush, double2* __restrict__ chi,
                   int* __restrict__ err, const GemmArgs ga, const Ctl ctl) {
  using C = Cfg<TERMS, BK, STAGES, FUSED>;
  constexpr int TILE_BYTES = C::TILE_BYTES;
  constexpr int AST = C::AST;
  static_assert(!FUSED || (TERMS == 2 && BK == 64 && !GEMM), "fused weighting: two terms, 64-element stages");
  static_assert(CL == 1 || (CL == 2 && !GEMM && !FUSED), "B multicast: the stored-operand rank-k form only");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::RING_BYTES);  // stage (fused: B rows) landed
  uint64_t* empty = full + 4;   // stage consumed by the MMAs
  uint64_t* conv = empty + 4;   // fused: A stage converted (A hi/lo tiles ready)
  uint64_t* fullA = conv + 4;   // fused: the FP32 A rows of the A stage landed
  uint64_t* emptyA = fullA + 4; // fused: A stage consumed by the MMAs
  uint64_t* tfull = emptyA + 4;
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
  const uint64_t wait_ns = ctl.wait_ns;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], CL);
    }
    for (int s = 0; s < AST; ++s) {
      mbar_init(&conv[s], CONV_WARPS);
      mbar_init(&fullA[s], 1);
      mbar_init(&emptyA[s], 1);
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
  // the peer's barriers are initialised before any multicast reaches them
  if constexpr (CL > 1) cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int issued = 0, issuedA = 0;
      for (int kb = 0; kb < nk; ++kb) {
        // test hook: withhold this stage, so the consumers' bounded waits run out
        if (kb == ctl.stall_stage) break;
        // HERK: A rows w * NGpad + i0 (weighted per frequency), X / Z rows j0;
        // fused: the FP32 rows i0 of F (both 32-float halves of the K block);
        // GEMM: A rows i0 (pairs), X / Z rows wk * NGpad + j0 of frequency wk
        const int wk = GEMM ? kb / ga.nkw : 0;
        const int k = GEMM ? (kb - wk * ga.nkw) * BK : kb * BK;
        const int arow = GEMM ? i0 : w * NGpad + i0;
        const int brow = GEMM ? (w * ga.nwb + wk) * NGpad + j0 : j0;
        if constexpr (FUSED) {
          // the A rows first, into their own deeper ring: issued as soon as
          // the MMAs of stage kb - AST are done, two stages ahead of use
          const int sa = kb % AST;
          if (kb >= AST && !mbar_wait(&emptyA[sa], ((kb / AST) & 1) ^ 1, abort_flag, wait_ns)) {
            *abort_flag = 1;
            atomicExch(err, 1);
            break;
          }
          unsigned char* at = C::a_ptr(smem, sa);
          mbar_expect_tx(&fullA[sa], 2 * TILE_BYTES);
          tma_load_2d(at, &maps.a[0], &fullA[sa], k, i0);
          tma_load_2d(at + TILE_BYTES, &maps.a[0], &fullA[sa], k + 32, i0);
          issuedA = kb + 1;
        }
        const int s = kb % STAGES;
        if (kb >= STAGES && !mbar_wait(&empty[s], ((kb / STAGES) & 1) ^ 1, abort_flag, wait_ns)) {
          *abort_flag = 1;
          atomicExch(err, 1);
          break;
        }
        if constexpr (FUSED) {
          mbar_expect_tx(&full[s], C::B_BYTES);
        } else {
          mbar_expect_tx(&full[s], C::STAGE_BYTES);
          unsigned char* at = C::a_ptr(smem, s);
#pragma unroll
          for (int t = 0; t < TERMS; ++t) tma_load_2d(at + t * TILE_BYTES, &maps.a[t], &full[s], k, arow);
        }
        unsigned char* bt = C::b_ptr(smem, s);
        if constexpr (CL > 1) {
          // rank 0 the X tiles, rank 1 the Z tiles, each for both CTAs
          const uint32_t r = cluster_rank();
#pragma unroll
          for (int t = 0; t < TERMS; ++t)
            tma_load_2d_mc(bt + (2 * t + r) * TILE_BYTES, r ? &maps.z[t] : &maps.x[t], &full[s], k, brow, 0x3);
        } else {
#pragma unroll
          for (int t = 0; t < TERMS; ++t) {
            tma_load_2d(bt + (2 * t) * TILE_BYTES, &maps.x[t], &full[s], k, brow);
            tma_load_2d(bt + (2 * t + 1) * TILE_BYTES, &maps.z[t], &full[s], k, brow);
          }
        }
        issued = kb + 1;
      }
      // pair: both CTAs' products have released the last issued slots, so no
      // arrival from the peer is still on its way to this CTA's barriers
      if constexpr (CL > 1) {
        for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
          if (!mbar_wait_timer(&empty[kb % STAGES], (kb / STAGES) & 1)) atomicExch(err, 7);
      }
      // every load already issued must land before the CTA may exit, also when
      // another role aborts after this loop ended: the last STAGES (AST)
      // issued stages hold distinct slots, and without an abort the consumers
      // have already seen them land, so these waits return at once
      for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
        if (!mbar_wait_timer(&full[kb % STAGES], (kb / STAGES) & 1)) atomicExch(err, 7);
      for (int kb = (issuedA > AST ? issuedA - AST : 0); kb < issuedA; ++kb)
        if (!mbar_wait_timer(&fullA[kb % AST], (kb / AST) & 1)) atomicExch(err, 7);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      // N = 256: the B operand is X (rows 0-127, giving Re) stacked on Z
      // (rows 128-255, giving Im), so one MMA fills both accumulators
      constexpr uint32_t idesc = idesc_bf16(BM, 2 * BN);
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        const int sa = FUSED ? kb % AST : s;
        // fused: the converters' barrier (A tiles), then the B rows
        if ((FUSED && !mbar_wait(&conv[sa], (kb / AST) & 1, abort_flag, wait_ns)) ||
            !mbar_wait(&full[s], (kb / STAGES) & 1, abort_flag, wait_ns)) {
          *abort_flag = 1;
          atomicExch(err, 2);
          break;
        }
        const int f = kb / fold;
        const int b = f & 1;
        const bool first = (kb % fold) == 0;
        if (first && f >= 2 && !mbar_wait(&tempty[b], ((f >> 1) - 1) & 1, abort_flag, wait_ns)) {
          *abort_flag = 1;
          atomicExch(err, 3);
          break;
        }
        tc_fence_after();
        const uint32_t sta = smem_u32(C::a_ptr(smem, sa));
        const uint32_t stb = smem_u32(C::b_ptr(smem, s));
        const uint32_t d = tmem + b * 256;  // Re in columns 0-127, Im in 128-255
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint32_t koff = kk * 32;  // 16 bf16 = 32 bytes along K inside the swizzle atom
          uint64_t da[3], db[3];
#pragma unroll
          for (int t = 0; t < TERMS; ++t) {
            da[t] = kmajor_desc<BK>(sta + t * TILE_BYTES + koff);
            db[t] = kmajor_desc<BK>(stb + (2 * t) * TILE_BYTES + koff);
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
        if constexpr (CL > 1)
          umma_commit_mc(&empty[s], 0x3);
        else
          umma_commit(&empty[s]);
        if (FUSED) umma_commit(&emptyA[sa]);
        if ((kb % fold) == fold - 1 || kb == nk - 1) umma_commit(&tfull[b]);
      }
      // every MMA issued so far must finish before TMEM is released
      umma_commit(mma_done);
      if (!mbar_wait_timer(mma_done, 0)) atomicExch(err, 5);
    }
  } else if (warp < EPI_WARP0) {
    // ------------------------------------------------------------ converters (fused weighting)
    // Thread ct handles 16-byte chunk c = ct % 8 of rows rb, rb + 8, ... of
    // both halves: four pairs of the stage, scaled by w_p(w) of this CTA's
    // frequency and split into bfloat16 hi (written over half 0) and lo
    // (written over half 1).  The same FP32 product and split as the
    // per-frequency preparation, so chi0 is bit-identical to that form.
    if constexpr (FUSED) {
      constexpr int CONV_ROWS = 32 * CONV_WARPS / 8;  // rows per pass: 8 chunks a row
      const int ct = threadIdx.x - 64;
      const int c = ct & 7, rb = ct >> 3;
      const float* wrow = ctl.wpad + (int64_t)w * ctl.wstride;
      for (int kb = 0; kb < nk; ++kb) {
        const int sa = kb % AST;
        if (!warp_wait(&fullA[sa], (kb / AST) & 1, abort_flag, wait_ns)) {
          *abort_flag = 1;
          atomicExch(err, 6);
          break;
        }
        const float4 wv = __ldg(reinterpret_cast<const float4*>(wrow + (int64_t)kb * 32 + 4 * c));
        unsigned char* t0 = C::a_ptr(smem, sa);
        unsigned char* t1 = t0 + TILE_BYTES;
#pragma unroll 4
        for (int j = 0; j < BM / CONV_ROWS; ++j) {
          const int g = rb + CONV_ROWS * j;
          const int off = g * 128 + ((c ^ (g & 7)) << 4);
          const float4 a = *reinterpret_cast<const float4*>(t0 + off);  // pairs 4c, 4c+1 (re, im)
          const float4 q = *reinterpret_cast<const float4*>(t1 + off);  // pairs 4c+2, 4c+3
          uint4 hi, lo;
          split_pair(__fmul_rn(wv.x, a.x), __fmul_rn(wv.x, a.y), hi.x, lo.x);
          split_pair(__fmul_rn(wv.y, a.z), __fmul_rn(wv.y, a.w), hi.y, lo.y);
          split_pair(__fmul_rn(wv.z, q.x), __fmul_rn(wv.z, q.y), hi.z, lo.z);
          split_pair(__fmul_rn(wv.w, q.z), __fmul_rn(wv.w, q.w), hi.w, lo.w);
          *reinterpret_cast<uint4*>(t0 + off) = hi;
          *reinterpret_cast<uint4*>(t1 + off) = lo;
        }
        // the tensor cores read shared memory through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&conv[sa]);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 4..19)
    // Warp w reads TMEM lane quarter w % 4 (rows 32q..32q+31) and column
    // slice cs (32 columns) of the Re and Im accumulators; four warps per
    // quarter drain a fold in a quarter of the time one would.  The FP32
    // partial of every fold is added to FP32 running sums held in registers
    // (round to nearest) and the running sums go to the FP64 chi0 every
    // `flush` folds, so the truncating accumulation inside the tensor core
    // never spans more than one fold.  A warp whose 32 rows are all padding,
    // or whose 32 columns all lie above the diagonal (or past the sphere),
    // writes nothing and skips its loads; it still keeps the fold protocol.
    const int q = warp & 3;
    const int cs = (warp - EPI_WARP0) >> 2;
    const int row = q * 32 + lane;
    const int gi = i0 + row;
    const int cbase = cs * 32;
    const int rlo = i0 + q * 32;
    bool active;
    if constexpr (GEMM)
      active = rlo < ga.P && j0 + cbase < NG;
    else
      active = rlo < NG && j0 + cbase < NG && j0 + cbase <= rlo + 31;
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
      if (!warp_wait(&tfull[b], (f >> 1) & 1, abort_flag, wait_ns)) {
        *abort_flag = 1;
        atomicExch(err, 4);
        break;
      }
      if (!active) {
        tc_fence_before();
        mbar_arrive(&tempty[b]);
        continue;
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
      // 20 warps leave 96 registers a thread: 64 running sums and one
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
    if (active) {
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
    }
#undef RPA_TC_FLUSH
  }
  tc_fence_before();
  __syncthreads();
  // neither CTA of a pair exits while the other may still address it
  if constexpr (CL > 1) cluster_sync_all();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ---------------------------------------------------------------- two-SM rank-k update
// The stored-operand two-term form on CTA pairs (cta_group::2).  A pair is the
// row tiles 2r (even CTA) and 2r + 1 (odd CTA) of one column tile and
// frequency; one thread of the even CTA issues M = 256, N = 256, K = 16
// products whose A rows come from both CTAs (128 each) and whose B operand is
// split the same way: the even CTA holds the X rows (Re), the odd CTA the Z
// rows (Im).  Each SM therefore stages and feeds the tensor core with half of
// B, which leaves room for three 64 KB stages.  Every CTA loads its own tiles
// and completes their bytes on the even CTA's stage barrier; the product
// commits arrive on the stage and accumulator barriers of both CTAs, and each
// CTA drains its own 128 accumulator rows.  Products, folds and flushes per
// element are those of herk_tc_kernel.
namespace tc2 {
constexpr int BK = 64, STAGES = 3, TERMS = 2;
constexpr int TILE_BYTES = BM * BK * 2;
constexpr int STAGE_BYTES = 2 * TERMS * TILE_BYTES;  // A hi, lo; B half hi, lo
constexpr int RING_BYTES = STAGES * STAGE_BYTES;
constexpr int SMEM_BYTES = RING_BYTES + 1024 + 256;
}  // namespace tc2

__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
// the tile lands in this CTA; its bytes complete on the barrier at cluster address bar
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, uint32_t bar, int k, int row) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(k), "r"(row)
      : "memory");
}
__device__ __forceinline__ void umma2(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma2_commit_both(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"((uint16_t)0x3)
      : "memory");
}
__device__ __forceinline__ void umma2_commit_local(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// arrive on a barrier of this CTA or its peer (cluster address); the ordering
// the accumulator hand-back needs is the completed tensor-memory loads
// (tcgen05.wait::ld and the fence before it), so CTA-scope release suffices
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}

// pair tile pt -> row pair r and column tile tj (tj <= 2r + 1, tj < nt)
__device__ __forceinline__ void pair_tile(int pt, int nt, int& r, int& tj) {
  r = 0;
  while (true) {
    const int cnt = min(2 * r + 2, nt);
    if (pt < cnt) break;
    pt -= cnt;
    ++r;
  }
  tj = pt;
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    herk_tc2_kernel(const __grid_constant__ Maps maps, int NG, int NGpad, int nk, int fold, int flush,
                    double2* __restrict__ chi, int* __restrict__ err, const Ctl ctl) {
  using namespace tc2;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + RING_BYTES);  // even CTA: stage landed in both
  uint64_t* empty = full + 4;                                      // stage consumed (both CTAs)
  uint64_t* tfull = empty + 4;                                     // accumulator buffer ready (both CTAs)
  uint64_t* tempty = tfull + 2;                                    // even CTA: buffer drained by both
  uint64_t* mma_done = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const int w = blockIdx.y;
  int rp, tj;
  pair_tile(blockIdx.x >> 1, NGpad / BM, rp, tj);
  const int ti = 2 * rp + (int)rank;
  const int i0 = ti * BM, j0 = tj * BN;
  const int nfold = (nk + fold - 1) / fold;
  const uint64_t wait_ns = ctl.wait_ns;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 2 * EPI_WARPS);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    // one warp of each CTA of the pair allocates the same columns in both
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer (both CTAs)
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < nk; ++kb) {
        if (kb == ctl.stall_stage) break;
        const int s = kb % STAGES;
        if (kb >= STAGES && !mbar_wait(&empty[s], ((kb / STAGES) & 1) ^ 1, abort_flag, wait_ns)) {
          *abort_flag = 1;
          atomicExch(err, 1);
          break;
        }
        if (rank == 0) mbar_expect_tx(&full[s], 2 * STAGE_BYTES);
        const uint32_t fb = peer_addr(&full[s], 0);
        unsigned char* st = smem + s * STAGE_BYTES;
        const int k = kb * BK;
#pragma unroll
        for (int t = 0; t < TERMS; ++t) {
          tma_load_2d_pair(st + t * TILE_BYTES, &maps.a[t], fb, k, w * NGpad + i0);
          tma_load_2d_pair(st + (TERMS + t) * TILE_BYTES, rank ? &maps.z[t] : &maps.x[t], fb, k, j0);
        }
        issued = kb + 1;
      }
      // the even CTA's loads and products must land before it may exit; both
      // wait until the pair's products released the last issued slots
      if (rank == 0)
        for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
          if (!mbar_wait_timer(&full[kb % STAGES], (kb / STAGES) & 1)) atomicExch(err, 7);
      for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
        if (!mbar_wait_timer(&empty[kb % STAGES], (kb / STAGES) & 1)) atomicExch(err, 7);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer (even CTA)
    if (lane == 0 && rank == 0) {
      constexpr uint32_t idesc = idesc_bf16(2 * BM, 2 * BN);
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        if (!mbar_wait(&full[s], (kb / STAGES) & 1, abort_flag, wait_ns)) {
          *abort_flag = 1;
          atomicExch(err, 2);
          break;
        }
        const int f = kb / fold;
        const int b = f & 1;
        const bool first = (kb % fold) == 0;
        if (first && f >= 2 && !mbar_wait(&tempty[b], ((f >> 1) - 1) & 1, abort_flag, wait_ns)) {
          *abort_flag = 1;
          atomicExch(err, 3);
          break;
        }
        tc_fence_after();
        const uint32_t st = smem_u32(smem + s * STAGE_BYTES);
        const uint32_t d = tmem + b * 256;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint32_t koff = kk * 32;
          const uint64_t a0 = kmajor_desc<BK>(st + koff), a1 = kmajor_desc<BK>(st + TILE_BYTES + koff);
          const uint64_t b0 = kmajor_desc<BK>(st + 2 * TILE_BYTES + koff);
          const uint64_t b1 = kmajor_desc<BK>(st + 3 * TILE_BYTES + koff);
          const uint32_t acc = (first && kk == 0) ? 0u : 1u;
          umma2(d, a0, b0, idesc, acc);  // hi*hi
          umma2(d, a0, b1, idesc, 1u);   // hi*lo
          umma2(d, a1, b0, idesc, 1u);   // lo*hi
        }
        umma2_commit_both(&empty[s]);
        if ((kb % fold) == fold - 1 || kb == nk - 1) umma2_commit_both(&tfull[b]);
      }
      umma2_commit_local(mma_done);
      if (!mbar_wait_timer(mma_done, 0)) atomicExch(err, 5);
    }
  } else if (warp >= EPI_WARP0) {
    // ------------------------------------------------------------ epilogue (both CTAs, own rows)
    const int q = warp & 3;
    const int cs = (warp - EPI_WARP0) >> 2;
    const int row = q * 32 + lane;
    const int gi = i0 + row;
    const int cbase = cs * 32;
    const int rlo = i0 + q * 32;
    const bool active = rlo < NG && j0 + cbase < NG && j0 + cbase <= rlo + 31;
    double2* crow = chi + ((int64_t)w * NG + gi) * NG + j0 + cbase;
    const int ncol = (gi < NG) ? max(0, min(32, min(NG, gi + 1) - (j0 + cbase))) : 0;
    float sre[32], sim[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) sre[c] = sim[c] = 0.f;
#define RPA_TC2_FLUSH()                                     \
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
    for (int f = 0; f < nfold; ++f) {
      const int b = f & 1;
      if (!warp_wait(&tfull[b], (f >> 1) & 1, abort_flag, wait_ns)) {
        *abort_flag = 1;
        atomicExch(err, 4);
        break;
      }
      // one arrival per warp on the even CTA's barrier, after every lane's loads
      if (!active) {
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(peer_addr(&tempty[b], 0));
        continue;
      }
      tc_fence_after();
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + b * 256 + cbase;
      float v[16];
      tmem_ld16(base, v);
#pragma unroll
      for (int c = 0; c < 16; ++c) sre[c] = fmaf(1.f, v[c], sre[c]);
      tmem_ld16(base + 16, v);
#pragma unroll
      for (int c = 0; c < 16; ++c) sre[16 + c] = fmaf(1.f, v[c], sre[16 + c]);
      tmem_ld16(base + 128, v);
#pragma unroll
      for (int c = 0; c < 16; ++c) sim[c] = fmaf(1.f, v[c], sim[c]);
      tmem_ld16(base + 144, v);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(peer_addr(&tempty[b], 0));
#pragma unroll
      for (int c = 0; c < 16; ++c) sim[16 + c] = fmaf(1.f, v[c], sim[16 + c]);
      if ((f + 1) % flush == 0) RPA_TC2_FLUSH();
    }
    if (active) RPA_TC2_FLUSH();
#undef RPA_TC2_FLUSH
  }
  tc_fence_before();
  __syncthreads();
  // neither CTA exits (or frees its tensor memory) while the other may still address it
  cluster_sync_all();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ---------------------------------------------------------------- persistent batched launch
// Many rank-k blocks (k-blocks of several q-points and instances, each with
// its own operands and K) in one persistent launch of two-term tiles.  A
// unit is one chi (one q-point of one instance) with the blocks that add to
// it; a work item is (unit, lower-triangle tile, frequency) and runs the
// unit's blocks one after another, so no two CTAs ever add to the same chi
// element.  One CTA per SM pulls items from a device counter; the load role
// takes each item and publishes it in a four-slot shared ring that the MMA,
// converter and epilogue roles read in the same order (each consumer warp
// releases the slot once it has read it).  The stage and fold counters run on
// across items, so the shared-memory rings and the two TMEM accumulators stay
// in flight from one item to the next.  Per block the arithmetic is that of
// herk_tc_kernel (same products, folds and flushes, blocks in the same
// order), so chi0 is bit-identical to one launch per block.
constexpr int BATCH_MAX_JOBS = 24;
constexpr int BATCH_MAX_UNITS = 24;
constexpr int ITEM_SLOTS = 4;

struct BatchJob {
  CUtensorMap a[2];    // unfused: weighted A terms (rows w NGpad + i); fused: a[0] = F
  CUtensorMap x[2];
  CUtensorMap z[2];
  const float* wpad;   // fused: weights [nw][wstride]
  int64_t wstride;
  int nk;              // K stages
};

struct BatchUnit {
  double2* chi;        // [nw][NG][NG], lower triangle accumulated
  int item0;           // first item; the unit's items are tile + ntile * w
  int job0, njob;      // its blocks, in order
  int NG, NGpad, ntile;
};

struct BatchArgs {
  BatchJob job[BATCH_MAX_JOBS];
  BatchUnit unit[BATCH_MAX_UNITS];
  int nunits;
  int nitems;
  int* queue;          // item counter, zero at launch
  int fold, flush;
  uint64_t wait_ns;
};

__device__ __forceinline__ int batch_unit_of(const BatchArgs& ba, int item) {
  int u = 0;
  while (u + 1 < ba.nunits && item >= ba.unit[u + 1].item0) ++u;
  return u;
}

template <bool FUSED>
__global__ void __launch_bounds__(NUM_THREADS, 1) herk_tc_batch_kernel(const __grid_constant__ BatchArgs ba,
                                                                        int* __restrict__ err) {
  using C = Cfg<2, 64, 2, FUSED>;
  constexpr int TERMS = 2, BK = 64, STAGES = 2;
  constexpr int TILE_BYTES = C::TILE_BYTES;
  constexpr int AST = C::AST;
  constexpr int CONSUMERS = 1 + (FUSED ? CONV_WARPS : 0) + EPI_WARPS;  // warps that read every item
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::RING_BYTES);
  uint64_t* empty = full + 4;
  uint64_t* conv = empty + 4;
  uint64_t* fullA = conv + 4;
  uint64_t* emptyA = fullA + 4;
  uint64_t* tfull = emptyA + 4;
  uint64_t* tempty = tfull + 2;
  uint64_t* mma_done = tempty + 2;
  uint64_t* ifull = mma_done + 1;        // item slot published
  uint64_t* iempty = ifull + ITEM_SLOTS; // item slot read by every consumer warp
  volatile int* islot = reinterpret_cast<volatile int*>(iempty + ITEM_SLOTS);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(iempty + ITEM_SLOTS) + ITEM_SLOTS;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t wait_ns = ba.wait_ns;
  const int fold = ba.fold;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < AST; ++s) {
      mbar_init(&conv[s], CONV_WARPS);
      mbar_init(&fullA[s], 1);
      mbar_init(&emptyA[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 32 * EPI_WARPS);
    }
    mbar_init(mma_done, 1);
    for (int r = 0; r < ITEM_SLOTS; ++r) {
      mbar_init(&ifull[r], 1);
      mbar_init(&iempty[r], CONSUMERS);
    }
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
    // ------------------------------------------------------------ items and TMA loads
    if (lane == 0) {
      int64_t issued = 0, issuedA = 0;  // stages whose B (A) rows were issued, over all items
      bool stop = false;
      for (int seq = 0; !stop; ++seq) {
        const int r = seq % ITEM_SLOTS;
        if (seq >= ITEM_SLOTS && !mbar_wait(&iempty[r], ((seq / ITEM_SLOTS) & 1) ^ 1, abort_flag, wait_ns)) {
          stop = true;
          break;
        }
        const int item = atomicAdd(ba.queue, 1);
        const bool done = item >= ba.nitems;
        islot[r] = done ? -1 : item;
        mbar_arrive(&ifull[r]);
        if (done) break;
        const BatchUnit& U = ba.unit[batch_unit_of(ba, item)];
        const int local = item - U.item0;
        const int w = local / U.ntile;
        int ti, tj;
        tri_tile(local - w * U.ntile, ti, tj);
        const int i0 = ti * BM, j0 = tj * BN;
        for (int jb = U.job0; jb < U.job0 + U.njob && !stop; ++jb) {
          const BatchJob& J = ba.job[jb];
          for (int kb = 0; kb < J.nk; ++kb) {
            const int64_t g = issued;  // global stage index of this stage
            const int k = kb * BK;
            if constexpr (FUSED) {
              const int sa = (int)(g % AST);
              if (g >= AST && !mbar_wait(&emptyA[sa], ((g / AST) & 1) ^ 1, abort_flag, wait_ns)) {
                stop = true;
                break;
              }
              unsigned char* at = C::a_ptr(smem, sa);
              mbar_expect_tx(&fullA[sa], 2 * TILE_BYTES);
              tma_load_2d(at, &J.a[0], &fullA[sa], k, i0);
              tma_load_2d(at + TILE_BYTES, &J.a[0], &fullA[sa], k + 32, i0);
              issuedA = g + 1;
            }
            const int s = (int)(g % STAGES);
            if (g >= STAGES && !mbar_wait(&empty[s], ((g / STAGES) & 1) ^ 1, abort_flag, wait_ns)) {
              stop = true;
              break;
            }
            if constexpr (FUSED) {
              mbar_expect_tx(&full[s], C::B_BYTES);
            } else {
              mbar_expect_tx(&full[s], C::STAGE_BYTES);
              unsigned char* at = C::a_ptr(smem, s);
#pragma unroll
              for (int t = 0; t < TERMS; ++t)
                tma_load_2d(at + t * TILE_BYTES, &J.a[t], &full[s], k, w * U.NGpad + i0);
            }
            unsigned char* bt = C::b_ptr(smem, s);
#pragma unroll
            for (int t = 0; t < TERMS; ++t) {
              tma_load_2d(bt + (2 * t) * TILE_BYTES, &J.x[t], &full[s], k, j0);
              tma_load_2d(bt + (2 * t + 1) * TILE_BYTES, &J.z[t], &full[s], k, j0);
            }
            issued = g + 1;
          }
        }
      }
      if (stop) {
        *abort_flag = 1;
        atomicExch(err, 1);
      }
      // every load already issued must land before the CTA may exit
      for (int64_t g = (issued > STAGES ? issued - STAGES : 0); g < issued; ++g)
        if (!mbar_wait_timer(&full[g % STAGES], (g / STAGES) & 1)) atomicExch(err, 7);
      for (int64_t g = (issuedA > AST ? issuedA - AST : 0); g < issuedA; ++g)
        if (!mbar_wait_timer(&fullA[g % AST], (g / AST) & 1)) atomicExch(err, 7);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(BM, 2 * BN);
      int64_t gs = 0, gf = 0;  // stages and folds consumed, over all items
      bool stop = false;
      for (int seq = 0; !stop; ++seq) {
        const int r = seq % ITEM_SLOTS;
        if (!mbar_wait(&ifull[r], (seq / ITEM_SLOTS) & 1, abort_flag, wait_ns)) {
          stop = true;
          break;
        }
        const int item = islot[r];
        mbar_arrive(&iempty[r]);
        if (item < 0) break;
        const BatchUnit& U = ba.unit[batch_unit_of(ba, item)];
        for (int jb = U.job0; jb < U.job0 + U.njob && !stop; ++jb) {
          const int nk = ba.job[jb].nk;
          for (int kb = 0; kb < nk; ++kb) {
            const int64_t g = gs + kb;
            const int s = (int)(g % STAGES);
            const int sa = FUSED ? (int)(g % AST) : s;
            if ((FUSED && !mbar_wait(&conv[sa], (g / AST) & 1, abort_flag, wait_ns)) ||
                !mbar_wait(&full[s], (g / STAGES) & 1, abort_flag, wait_ns)) {
              stop = true;
              break;
            }
            const int64_t f = gf + kb / fold;
            const int b = (int)(f & 1);
            const bool first = (kb % fold) == 0;
            if (first && f >= 2 && !mbar_wait(&tempty[b], ((f >> 1) - 1) & 1, abort_flag, wait_ns)) {
              stop = true;
              break;
            }
            tc_fence_after();
            const uint32_t sta = smem_u32(C::a_ptr(smem, sa));
            const uint32_t stb = smem_u32(C::b_ptr(smem, s));
            const uint32_t d = tmem + b * 256;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint32_t koff = kk * 32;
              const uint64_t da0 = kmajor_desc<BK>(sta + koff), da1 = kmajor_desc<BK>(sta + TILE_BYTES + koff);
              const uint64_t db0 = kmajor_desc<BK>(stb + koff), db1 = kmajor_desc<BK>(stb + 2 * TILE_BYTES + koff);
              umma(d, da0, db0, idesc, (first && kk == 0) ? 0u : 1u);
              umma(d, da0, db1, idesc, 1u);
              umma(d, da1, db0, idesc, 1u);
            }
            umma_commit(&empty[s]);
            if (FUSED) umma_commit(&emptyA[sa]);
            if ((kb % fold) == fold - 1 || kb == nk - 1) umma_commit(&tfull[b]);
          }
          gs += nk;
          gf += (nk + fold - 1) / fold;
        }
      }
      if (stop) {
        *abort_flag = 1;
        atomicExch(err, 2);
      }
      umma_commit(mma_done);
      if (!mbar_wait_timer(mma_done, 0)) atomicExch(err, 5);
    }
  } else if (warp < EPI_WARP0) {
    // ------------------------------------------------------------ converters (fused weighting)
    if constexpr (FUSED) {
      constexpr int CONV_ROWS = 32 * CONV_WARPS / 8;
      const int ct = threadIdx.x - 64;
      const int c = ct & 7, rb = ct >> 3;
      int gs = 0;
      bool stop = false;
      for (int seq = 0; !stop; ++seq) {
        const int r = seq % ITEM_SLOTS;
        if (!warp_wait(&ifull[r], (seq / ITEM_SLOTS) & 1, abort_flag, wait_ns)) {
          stop = true;
          break;
        }
        const int item = islot[r];
        __syncwarp();
        if (lane == 0) mbar_arrive(&iempty[r]);
        if (item < 0) break;
        const BatchUnit& U = ba.unit[batch_unit_of(ba, item)];
        const int w = (item - U.item0) / U.ntile;
        for (int jb = U.job0; jb < U.job0 + U.njob && !stop; ++jb) {
          const BatchJob& J = ba.job[jb];
          const float* wrow = J.wpad + (int64_t)w * J.wstride;
          for (int kb = 0; kb < J.nk; ++kb) {
            const int g = gs + kb;
            const int sa = g % AST;
            if (!warp_wait(&fullA[sa], (g / AST) & 1, abort_flag, wait_ns)) {
              stop = true;
              break;
            }
            const float4 wv = __ldg(reinterpret_cast<const float4*>(wrow + (int64_t)kb * 32 + 4 * c));
            unsigned char* t0 = C::a_ptr(smem, sa);
            unsigned char* t1 = t0 + TILE_BYTES;
#pragma unroll 4
            for (int jr = 0; jr < BM / CONV_ROWS; ++jr) {
              const int gr = rb + CONV_ROWS * jr;
              const int off = gr * 128 + ((c ^ (gr & 7)) << 4);
              const float4 a = *reinterpret_cast<const float4*>(t0 + off);
              const float4 q = *reinterpret_cast<const float4*>(t1 + off);
              uint4 hi, lo;
              split_pair(__fmul_rn(wv.x, a.x), __fmul_rn(wv.x, a.y), hi.x, lo.x);
              split_pair(__fmul_rn(wv.y, a.z), __fmul_rn(wv.y, a.w), hi.y, lo.y);
              split_pair(__fmul_rn(wv.z, q.x), __fmul_rn(wv.z, q.y), hi.z, lo.z);
              split_pair(__fmul_rn(wv.w, q.z), __fmul_rn(wv.w, q.w), hi.w, lo.w);
              *reinterpret_cast<uint4*>(t0 + off) = hi;
              *reinterpret_cast<uint4*>(t1 + off) = lo;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&conv[sa]);
          }
          gs += J.nk;
        }
      }
      if (stop) {
        *abort_flag = 1;
        atomicExch(err, 6);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 4..19)
    const int q = warp & 3;
    const int cs = (warp - EPI_WARP0) >> 2;
    const int row = q * 32 + lane;
    const int cbase = cs * 32;
    int gf = 0;
    bool stop = false;
    for (int seq = 0; !stop; ++seq) {
      const int r = seq % ITEM_SLOTS;
      if (!warp_wait(&ifull[r], (seq / ITEM_SLOTS) & 1, abort_flag, wait_ns)) {
        stop = true;
        break;
      }
      const int item = islot[r];
      __syncwarp();
      if (lane == 0) mbar_arrive(&iempty[r]);
      if (item < 0) break;
      const BatchUnit& U = ba.unit[batch_unit_of(ba, item)];
      const int NG = U.NG;
      const int local = item - U.item0;
      const int w = local / U.ntile;
      int ti, tj;
      tri_tile(local - w * U.ntile, ti, tj);
      const int i0 = ti * BM, j0 = tj * BN;
      const int gi = i0 + row;
      const int rlo = i0 + q * 32;
      const bool active = rlo < NG && j0 + cbase < NG && j0 + cbase <= rlo + 31;
      double2* crow = U.chi + ((int64_t)w * NG + gi) * NG + j0 + cbase;
      const int ncol = (gi < NG) ? max(0, min(32, min(NG, gi + 1) - (j0 + cbase))) : 0;
      for (int jb = U.job0; jb < U.job0 + U.njob && !stop; ++jb) {
        const int nfold = (ba.job[jb].nk + fold - 1) / fold;
        float sre[32], sim[32];
#pragma unroll
        for (int cc = 0; cc < 32; ++cc) sre[cc] = sim[cc] = 0.f;
#define RPA_TCB_FLUSH()                                     \
  do {                                                      \
    _Pragma("unroll") for (int cc = 0; cc < 32; ++cc) {     \
      if (cc < ncol) {                                      \
        double2 v = crow[cc];                               \
        v.x += (double)sre[cc];                             \
        v.y += (double)sim[cc];                             \
        crow[cc] = v;                                       \
      }                                                     \
      sre[cc] = 0.f;                                        \
      sim[cc] = 0.f;                                        \
    }                                                       \
  } while (0)
        for (int f = 0; f < nfold; ++f) {
          const int F = gf + f;
          const int b = F & 1;
          if (!warp_wait(&tfull[b], (F >> 1) & 1, abort_flag, wait_ns)) {
            stop = true;
            break;
          }
          if (!active) {
            tc_fence_before();
            mbar_arrive(&tempty[b]);
            continue;
          }
          tc_fence_after();
          const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + b * 256 + cbase;
          float v[16];
          tmem_ld16(base, v);
#pragma unroll
          for (int cc = 0; cc < 16; ++cc) sre[cc] += v[cc];
          tmem_ld16(base + 16, v);
#pragma unroll
          for (int cc = 0; cc < 16; ++cc) sre[16 + cc] += v[cc];
          tmem_ld16(base + 128, v);
#pragma unroll
          for (int cc = 0; cc < 16; ++cc) sim[cc] += v[cc];
          tmem_ld16(base + 144, v);
          tc_fence_before();
          mbar_arrive(&tempty[b]);
#pragma unroll
          for (int cc = 0; cc < 16; ++cc) sim[16 + cc] += v[cc];
          // the last fold of each block flushes as well (one flush site keeps
          // the running sums in registers); after an abort nothing is flushed
          if ((f + 1) % ba.flush == 0 || f == nfold - 1) RPA_TCB_FLUSH();
        }
#undef RPA_TCB_FLUSH
        gf += nfold;
      }
    }
    if (stop) {
      *abort_flag = 1;
      atomicExch(err, 4);
    }
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

// The operand preparation runs on a second stream beside the rank-k kernel
// of the previous block.  That kernel leaves 4096 registers of an SM free
// (640 threads x 96), so the preparation uses 128-thread blocks of at most 32
// registers a thread, which fit beside it instead of waiting for its waves.
constexpr int PREP_ROWS = 4;                   // transpose rows per pass
constexpr int PREP_THREADS = 32 * PREP_ROWS;   // 128

// X[t][g][2p+c], Z[t][g][2p+c] from N[p][g] (transpose through shared memory), zero padding.
template <int TERMS>
__global__ void __launch_bounds__(PREP_THREADS, 16) prep_xz_kernel(const float2* __restrict__ N, int64_t P, int NG, int NGpad,
                                                      int64_t Kpad, __nv_bfloat162* __restrict__ X,
                                                      __nv_bfloat162* __restrict__ Z, int64_t term_stride) {
  __shared__ float2 t[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x PREP_ROWS
  const int64_t p0 = (int64_t)blockIdx.y * 32;
  const int g0 = blockIdx.x * 32;
  for (int r = ty; r < 32; r += PREP_ROWS) {
    const int64_t p = p0 + r;
    const int g = g0 + tx;
    t[r][tx] = (p < P && g < NG) ? N[p * NG + g] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += PREP_ROWS) {
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

// Fused weighting, two terms: X, Z as prep_xz_kernel<2>, plus F = the FP32
// (Re, Im) N[p][g] at row g, K position f_pos(2p) (zero padding), and the
// weights padded to wstride pairs per frequency (zero past the last pair).
__global__ void __launch_bounds__(PREP_THREADS, 16) prep_xzf_kernel(const float2* __restrict__ N, const float* __restrict__ wgt,
                                                       int64_t P, int NG, int64_t Kpad, int nw,
                                                       __nv_bfloat162* __restrict__ X, __nv_bfloat162* __restrict__ Z,
                                                       int64_t term_stride, float2* __restrict__ F,
                                                       float* __restrict__ wpad, int64_t wstride) {
  __shared__ float2 t[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x PREP_ROWS
  const int64_t p0 = (int64_t)blockIdx.y * 32;
  const int g0 = blockIdx.x * 32;
  for (int r = ty; r < 32; r += PREP_ROWS) {
    const int64_t p = p0 + r;
    const int g = g0 + tx;
    t[r][tx] = (p < P && g < NG) ? N[p * NG + g] : make_float2(0.f, 0.f);
  }
  if (blockIdx.x == 0)
    for (int w = ty; w < nw; w += PREP_ROWS) {
      const int64_t p = p0 + tx;
      wpad[(int64_t)w * wstride + p] = p < P ? wgt[(int64_t)w * P + p] : 0.f;
    }
  __syncthreads();
  // K position of pair p0 + tx inside its 64-element block (p0 is a multiple of 32)
  const int64_t fk = f_pos(2 * (p0 + tx));
  for (int r = ty; r < 32; r += PREP_ROWS) {
    const int g = g0 + r;
    const int64_t p = p0 + tx;
    const float2 v = t[tx][r];
    const int64_t o = (int64_t)g * (Kpad / 2) + p;
    __nv_bfloat16 rh, rl, ih, il;
    split2(v.x, rh, rl);
    split2(v.y, ih, il);
    X[o] = __halves2bfloat162(rh, ih);
    X[o + term_stride] = __halves2bfloat162(rl, il);
    Z[o] = __halves2bfloat162(__hneg(ih), rh);
    Z[o + term_stride] = __halves2bfloat162(__hneg(il), rl);
    F[((int64_t)g * Kpad + fk) / 2] = v;
  }
}

// A[t][w][g][2p+c] = split(w_p(w) * (Re, Im) N[p][g]) for every frequency.
template <int TERMS>
__global__ void __launch_bounds__(PREP_THREADS, 16) prep_a_kernel(const float2* __restrict__ N, const float* __restrict__ wgt,
                                                     int64_t P, int NG, int NGpad, int64_t Kpad, int nw,
                                                     __nv_bfloat162* __restrict__ A, int64_t term_stride) {
  __shared__ float2 t[32][33];
  __shared__ float ws[32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x PREP_ROWS
  const int64_t p0 = (int64_t)blockIdx.y * 32;
  const int g0 = blockIdx.x * 32;
  for (int r = ty; r < 32; r += PREP_ROWS) {
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
    for (int r = ty; r < 32; r += PREP_ROWS) {
      const int g = g0 + r;
      const float2 v = t[tx][r];
      const float wp = ws[tx];
      const int64_t o = ((int64_t)w * NGpad + g) * (Kpad / 2) + p0 + tx;
      __nv_bfloat16 rh, rm, rl, ih, im, il;
      // the product is rounded to FP32 before the split (never contracted
      // into the split's subtraction), as in the fused converters
      if (TERMS == 2) {
        split2(__fmul_rn(wp, v.x), rh, rl);
        split2(__fmul_rn(wp, v.y), ih, il);
        A[o] = __halves2bfloat162(rh, ih);
        A[o + term_stride] = __halves2bfloat162(rl, il);
      } else {
        split3(__fmul_rn(wp, v.x), rh, rm, rl);
        split3(__fmul_rn(wp, v.y), ih, im, il);
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

// Row-major [rows][K] matrix, boxes of bk elements x BM rows; bfloat16 boxes
// of 64 (128 bytes, 128-byte swizzle) or 32 elements (64-byte swizzle), FP32
// boxes of 32 elements (128 bytes, 128-byte swizzle).
static bool make_map(CUtensorMap* m, const void* base, int64_t K, int64_t rows, int bk, bool fp32 = false) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int es_bytes = fp32 ? 4 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(K * es_bytes)};
  cuuint32_t box[2] = {(cuuint32_t)bk, BM};
  cuuint32_t es[2] = {1, 1};
  const bool sw128 = bk * es_bytes == 128;
  CUresult r = fn(m, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  sw128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
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

// Scratch of one k-block.  Unfused: X terms, Z terms, then the
// per-frequency A terms.  Fused (two terms): X terms, Z terms, F (FP32), the
// padded weights.
size_t herk_tc_scratch_bytes(int64_t P, int NG, int nw, int terms, int fused) {
  const tc::Geometry g = tc::geometry(P, NG);
  const size_t op = (size_t)g.NGpad * g.Kpad * 2;  // one bf16 operand matrix
  if (fused && terms == 2) return op * 4 + op * 2 + (size_t)nw * g.Ppad * 4;
  return op * (size_t)terms * (size_t)(nw + 2);
}

template <int TERMS, int BK, int STAGES, bool FUSED>
static cudaError_t launch_gemm(const tc::Maps& maps, dim3 grid, int NG, int NGpad, int64_t Kpad, int fold64, int flush,
                               double2* chi, int* err, const tc::Ctl& ctl, cudaStream_t s, bool pair = false) {
  using namespace tc;
  using C = Cfg<TERMS, BK, STAGES, FUSED>;
  static_assert(C::SMEM_BYTES <= 227 * 1024, "shared-memory ring too large");
  const int nk = (int)(Kpad / BK);
  // the fold length counts 64-element units of three products (two terms);
  // with three terms (six products per element) a unit is 32 elements, so a
  // fold holds the same number of truncating tensor-core accumulations
  const int fold = TERMS == 3 ? fold64 * (32 / BK) : fold64 * (64 / BK);
  if constexpr (!FUSED && TERMS == 2 && BK == 64) {
    if (pair) {
      // clusters of two frequencies sharing the B tiles (grid.y even)
      if (grid.y % 2) return cudaErrorInvalidValue;
      auto kern = herk_tc_kernel<TERMS, BK, STAGES, false, false, 2>;
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
      if (e != cudaSuccess) return e;
      cudaLaunchConfig_t cfg;
      memset(&cfg, 0, sizeof(cfg));
      cfg.gridDim = grid;
      cfg.blockDim = dim3(NUM_THREADS);
      cfg.dynamicSmemBytes = C::SMEM_BYTES;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 1;
      attr[0].val.clusterDim.y = 2;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, kern, maps, NG, NGpad, nk, fold, flush, chi, err, GemmArgs{}, ctl);
    }
  }
  cudaError_t e = cudaFuncSetAttribute(herk_tc_kernel<TERMS, BK, STAGES, false, FUSED, 1>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  herk_tc_kernel<TERMS, BK, STAGES, false, FUSED, 1><<<grid, NUM_THREADS, C::SMEM_BYTES, s>>>(
      maps, NG, NGpad, nk, fold, flush, chi, err, GemmArgs{}, ctl);
  return cudaGetLastError();
}

// Bounds shared by the two calls below.
static cudaError_t check_args(int64_t P, int NG, int nw, int terms, int fused, size_t scratch_bytes) {
  if (terms != 2 && terms != 3) return cudaErrorInvalidValue;
  const tc::Geometry g = tc::geometry(P, NG);
  if (scratch_bytes < herk_tc_scratch_bytes(P, NG, nw, terms, fused)) return cudaErrorInvalidValue;
  if (g.Kpad > (int64_t)1 << 31 || (int64_t)nw * g.NGpad > (1 << 30)) return cudaErrorInvalidValue;
  return cudaSuccess;
}

struct Operands {
  __nv_bfloat16 *X, *Z, *A;
  float* F;
  float* wpad;
  int64_t op_elems;
};
static Operands operands(void* scratch, const tc::Geometry& g, int terms) {
  Operands o;
  o.op_elems = (int64_t)g.NGpad * g.Kpad;
  o.X = (__nv_bfloat16*)scratch;
  o.Z = o.X + o.op_elems * terms;
  o.A = o.Z + o.op_elems * terms;
  o.F = (float*)o.A;                // fused: in place of the A terms
  o.wpad = o.F + o.op_elems;
  return o;
}

cudaError_t herk_tc_prepare(const float2* N, int64_t P, int NG, const float* wgt, int nw, int terms, int fused,
                            void* scratch, size_t scratch_bytes, cudaStream_t s) {
  using namespace tc;
  if (P == 0 || NG == 0 || nw == 0) return cudaSuccess;
  fused = fused && terms == 2;
  cudaError_t e = check_args(P, NG, nw, terms, fused, scratch_bytes);
  if (e != cudaSuccess) return e;
  const Geometry g = geometry(P, NG);
  const Operands o = operands(scratch, g, terms);
  dim3 pg(g.NGpad / 32, (unsigned)(g.Ppad / 32));
  if (fused) {
    prep_xzf_kernel<<<pg, PREP_THREADS, 0, s>>>(N, wgt, P, NG, g.Kpad, nw, (__nv_bfloat162*)o.X, (__nv_bfloat162*)o.Z,
                                       o.op_elems / 2, (float2*)o.F, o.wpad, g.Ppad);
  } else if (terms == 3) {
    prep_xz_kernel<3><<<pg, PREP_THREADS, 0, s>>>(N, P, NG, g.NGpad, g.Kpad, (__nv_bfloat162*)o.X, (__nv_bfloat162*)o.Z,
                                         o.op_elems / 2);
    prep_a_kernel<3><<<pg, PREP_THREADS, 0, s>>>(N, wgt, P, NG, g.NGpad, g.Kpad, nw, (__nv_bfloat162*)o.A,
                                        o.op_elems * nw / 2);
  } else {
    prep_xz_kernel<2><<<pg, PREP_THREADS, 0, s>>>(N, P, NG, g.NGpad, g.Kpad, (__nv_bfloat162*)o.X, (__nv_bfloat162*)o.Z,
                                         o.op_elems / 2);
    prep_a_kernel<2><<<pg, PREP_THREADS, 0, s>>>(N, wgt, P, NG, g.NGpad, g.Kpad, nw, (__nv_bfloat162*)o.A,
                                        o.op_elems * nw / 2);
  }
  return cudaGetLastError();
}

// The two-SM form: clusters of two CTAs over row-tile pairs.
static cudaError_t launch_tc2(const tc::Maps& maps, int NG, int NGpad, int nw, int64_t Kpad, int fold, int flush,
                              double2* chi, int* err, const tc::Ctl& ctl, cudaStream_t s) {
  using namespace tc;
  const int nt = NGpad / BM;
  int npair = 0;
  for (int r = 0; 2 * r < nt; ++r) npair += std::min(2 * r + 2, nt);
  cudaError_t e = cudaFuncSetAttribute(herk_tc2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc2::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(2 * npair, nw);
  cfg.blockDim = dim3(NUM_THREADS);
  cfg.dynamicSmemBytes = tc2::SMEM_BYTES;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int nk = (int)(Kpad / tc2::BK);
  return cudaLaunchKernelEx(&cfg, herk_tc2_kernel, maps, NG, NGpad, nk, fold, flush, chi, err, ctl);
}

cudaError_t herk_tc_run(int64_t P, int NG, int nw, int terms, int fused, int fold_stages, int flush_folds, int pipe,
                        int pair, int64_t wait_us, int stall_stage, double2* chi, void* scratch, size_t scratch_bytes,
                        int* err, cudaStream_t s) {
  using namespace tc;
  if (P == 0 || NG == 0 || nw == 0) return cudaSuccess;
  fused = fused && terms == 2 && pipe == 0;
  cudaError_t e = check_args(P, NG, nw, terms, fused, scratch_bytes);
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
    if (!make_map(&maps.x[t], o.X + o.op_elems * t, g.Kpad, g.NGpad, bk) ||
        !make_map(&maps.z[t], o.Z + o.op_elems * t, g.Kpad, g.NGpad, bk))
      return cudaErrorInvalidValue;
    if (fused) {
      if (t == 0 && !make_map(&maps.a[0], o.F, g.Kpad, g.NGpad, 32, true)) return cudaErrorInvalidValue;
    } else if (!make_map(&maps.a[t], o.A + o.op_elems * nw * t, g.Kpad, (int64_t)nw * g.NGpad, bk)) {
      return cudaErrorInvalidValue;
    }
  }
  Ctl ctl;
  ctl.wait_ns = (uint64_t)wait_us * 1000ull;
  ctl.stall_stage = stall_stage;
  ctl.wpad = fused ? o.wpad : nullptr;
  ctl.wstride = g.Ppad;
  const int nt = g.NGpad / BM;
  dim3 grid(nt * (nt + 1) / 2, nw);
  if (terms == 3)
    return launch_gemm<3, 32, 3, false>(maps, grid, NG, g.NGpad, g.Kpad, fold_stages, flush_folds, chi, err, ctl, s);
  if (bk == 32)
    return launch_gemm<2, 32, 4, false>(maps, grid, NG, g.NGpad, g.Kpad, fold_stages, flush_folds, chi, err, ctl, s);
  if (fused)
    return launch_gemm<2, 64, 2, true>(maps, grid, NG, g.NGpad, g.Kpad, fold_stages, flush_folds, chi, err, ctl, s);
  if (pair == 2) return launch_tc2(maps, NG, g.NGpad, nw, g.Kpad, fold_stages, flush_folds, chi, err, ctl, s);
  return launch_gemm<2, 64, 2, false>(maps, grid, NG, g.NGpad, g.Kpad, fold_stages, flush_folds, chi, err, ctl, s,
                                      pair == 1 && nw % 2 == 0);
}

// Controls of the batched-product launches: the default wait limit, no stall.
static tc::Ctl gemm_ctl() {
  tc::Ctl c;
  c.wait_ns = tc::DRAIN_NS;
  c.stall_stage = -1;
  c.wpad = nullptr;
  c.wstride = 0;
  return c;
}

// ---------------------------------------------------------------- persistent batched launch (host)
// Jobs are the k-blocks prepared by herk_tc_prepare (two terms), each with its
// own scratch; job j adds to the chi of unit unit_of[j] (jobs of one unit are
// consecutive and share NG and nw).  Units with more K stages are queued
// first, so the long items start early and the short ones fill the tail.
int herk_tc_batch_max_jobs() { return tc::BATCH_MAX_JOBS < tc::BATCH_MAX_UNITS ? tc::BATCH_MAX_JOBS
                                                                              : tc::BATCH_MAX_UNITS; }

cudaError_t herk_tc_batch_run(int njobs, const int64_t* P, const int* NG, const int* nw, void* const* scratch,
                              const size_t* scratch_bytes, const int* unit_of, double2* const* chi, int fused,
                              int fold_stages, int flush_folds, int64_t wait_us, int* queue, int* err,
                              cudaStream_t s) {
  using namespace tc;
  if (njobs < 1) return cudaSuccess;
  if (njobs > BATCH_MAX_JOBS || !queue) return cudaErrorInvalidValue;
  static int sm_count = 0;
  if (!sm_count) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sm_count < 1) return e != cudaSuccess ? e : cudaErrorInvalidValue;
  }
  // units: runs of consecutive jobs with the same unit_of (empty blocks dropped)
  struct U { std::vector<int> jobs; int64_t stages = 0; };
  std::vector<U> units;
  for (int j = 0; j < njobs; ++j) {
    if (P[j] <= 0 || NG[j] <= 0 || nw[j] <= 0) continue;
    if (units.empty() || unit_of[units.back().jobs.back()] != unit_of[j]) units.push_back(U());
    units.back().jobs.push_back(j);
    units.back().stages += geometry(P[j], NG[j]).Kpad / 64;
  }
  if (units.empty()) return cudaSuccess;
  if ((int)units.size() > BATCH_MAX_UNITS) return cudaErrorInvalidValue;
  std::stable_sort(units.begin(), units.end(), [](const U& x, const U& y) { return x.stages > y.stages; });
  BatchArgs* ba = new BatchArgs;
  memset(ba, 0, sizeof(BatchArgs));
  int64_t items = 0;
  int nj = 0;
  for (const U& u : units) {
    const int j0 = u.jobs[0];
    BatchUnit& B = ba->unit[ba->nunits++];
    const int NGpad = (NG[j0] + BM - 1) / BM * BM;
    const int nt = NGpad / BM;
    B.chi = chi[j0];
    B.item0 = (int)items;
    B.job0 = nj;
    B.njob = (int)u.jobs.size();
    B.NG = NG[j0];
    B.NGpad = NGpad;
    B.ntile = nt * (nt + 1) / 2;
    items += (int64_t)B.ntile * nw[j0];
    for (int j : u.jobs) {
      bool ok = NG[j] == NG[j0] && nw[j] == nw[j0] && chi[j] == chi[j0] &&
                check_args(P[j], NG[j], nw[j], 2, fused, scratch_bytes[j]) == cudaSuccess;
      const Geometry g = geometry(P[j], NG[j]);
      const Operands o = operands(scratch[j], g, 2);
      BatchJob& J = ba->job[nj++];
      for (int t = 0; t < 2 && ok; ++t) {
        ok = make_map(&J.x[t], o.X + o.op_elems * t, g.Kpad, g.NGpad, 64) &&
             make_map(&J.z[t], o.Z + o.op_elems * t, g.Kpad, g.NGpad, 64);
        if (fused)
          ok = ok && (t > 0 || make_map(&J.a[0], o.F, g.Kpad, g.NGpad, 32, true));
        else
          ok = ok && make_map(&J.a[t], o.A + o.op_elems * nw[j] * t, g.Kpad, (int64_t)nw[j] * g.NGpad, 64);
      }
      if (!ok) {
        delete ba;
        return cudaErrorInvalidValue;
      }
      J.wpad = fused ? o.wpad : nullptr;
      J.wstride = g.Ppad;
      J.nk = (int)(g.Kpad / 64);
    }
  }
  if (items >= ((int64_t)1 << 31) - 1 - sm_count) {
    delete ba;
    return cudaErrorInvalidValue;
  }
  ba->nitems = (int)items;
  ba->queue = queue;
  ba->fold = fold_stages < 1 ? 1 : fold_stages;
  ba->flush = flush_folds < 1 ? 1 : flush_folds;
  ba->wait_ns = (uint64_t)wait_us * 1000ull;
  const int smem = (fused ? Cfg<2, 64, 2, true>::RING_BYTES : Cfg<2, 64, 2, false>::RING_BYTES) + 1024 + 512;
  static_assert(Cfg<2, 64, 2, true>::RING_BYTES + 1024 + 512 <= 227 * 1024, "batched kernel shared memory");
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    if (fused) {
      e = cudaFuncSetAttribute(herk_tc_batch_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e == cudaSuccess) herk_tc_batch_kernel<true><<<sm_count, NUM_THREADS, smem, s>>>(*ba, err);
    } else {
      e = cudaFuncSetAttribute(herk_tc_batch_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e == cudaSuccess) herk_tc_batch_kernel<false><<<sm_count, NUM_THREADS, smem, s>>>(*ba, err);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  delete ba;
  return e;
}

// *dst[i] |= *src for every context of a batch (the batched kernel's flag).
__global__ void or_flags_kernel(const int* __restrict__ src, int* const* __restrict__ dst, int n) {
  const int v = *src;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (v) atomicOr(dst[i], v);
}

cudaError_t launch_or_flags(const int* src, int* const* dst, int n, cudaStream_t s) {
  if (n < 1) return cudaSuccess;
  or_flags_kernel<<<1, 128, 0, s>>>(src, dst, n);
  return cudaGetLastError();
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
      tc::prep_xz_kernel<3><<<pg, tc::PREP_THREADS, 0, s>>>(Gw, NG, NG, NGpad, KN, X + off, Z + off, op);
    else
      tc::prep_xz_kernel<2><<<pg, tc::PREP_THREADS, 0, s>>>(Gw, NG, NG, NGpad, KN, X + off, Z + off, op);
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
    if ((e = cudaFuncSetAttribute(herk_tc_kernel<3, 32, 3, true, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  C::SMEM_BYTES)) != cudaSuccess)
      return e;
    herk_tc_kernel<3, 32, 3, true, false, 1><<<grid, NUM_THREADS, C::SMEM_BYTES, s>>>(maps, NG, NGpad, nk, 1, 1, nullptr, err,
                                                                           ga, gemm_ctl());
  } else {
    using C = Cfg<2, 64, 2>;
    if ((e = cudaFuncSetAttribute(herk_tc_kernel<2, 64, 2, true, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  C::SMEM_BYTES)) != cudaSuccess)
      return e;
    herk_tc_kernel<2, 64, 2, true, false, 1><<<grid, NUM_THREADS, C::SMEM_BYTES, s>>>(maps, NG, NGpad, nk, 1, 1, nullptr, err,
                                                                           ga, gemm_ctl());
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
    if ((e = cudaFuncSetAttribute(herk_tc_kernel<3, 32, 3, true, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  C::SMEM_BYTES)) != cudaSuccess)
      return e;
    herk_tc_kernel<3, 32, 3, true, false, 1><<<grid, NUM_THREADS, C::SMEM_BYTES, s>>>(maps, NG, NGpad, nk, 1, 1, nullptr, err,
                                                                           ga, gemm_ctl());
  } else {
    using C = Cfg<2, 64, 2>;
    if ((e = cudaFuncSetAttribute(herk_tc_kernel<2, 64, 2, true, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  C::SMEM_BYTES)) != cudaSuccess)
      return e;
    herk_tc_kernel<2, 64, 2, true, false, 1><<<grid, NUM_THREADS, C::SMEM_BYTES, s>>>(maps, NG, NGpad, nk, 1, 1, nullptr, err,
                                                                           ga, gemm_ctl());
  }
  return cudaGetLastError();
}

}  // namespace rpa
