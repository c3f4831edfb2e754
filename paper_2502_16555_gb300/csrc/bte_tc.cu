// Tensor-core (tcgen05, sm_103a) trailing update of the FP32 per-point LU: A22 -= L21 U12 for every
// point of the batch, with the three-product TF32 split (a = a_hi + a_lo, b = b_hi + b_lo,
// ab ~ a_hi b_hi + a_hi b_lo + a_lo b_hi) accumulated in FP32 in tensor memory. This is the
// bulk O(Nv^3) work of the velocity-space solves of eq. "vspace_batched_system" (arXiv 2502.16555).
//
// Operands: the panel kernel writes L21 split into hi/lo parts, and the swap/TRSM kernel writes
// U12 transposed and split, into a workspace laid out K-major ([point][row][128] floats), so both
// MMA operands are K-major, 128-byte-swizzled TMA tiles.
//
// Kernel: persistent, one CTA of 192 threads per SM, static round-robin over 128x128 output tiles
// (point-major, so the CTAs in flight share one point's panels in L2):
//   warp 0  TMA producer: per K-chunk of 32, four 16 KB boxes (A_hi, A_lo, B_hi, B_lo) into a
//           3-stage shared-memory ring, completion through mbarrier transaction counts;
//   warp 1  allocates 256 TMEM columns (two 128x128 FP32 accumulators) and issues the MMAs
//           (M=128, N=128, K=8 per instruction, 12 per chunk), committing each stage back to the
//           producer and each finished accumulator to the epilogue;
//   warps 2-5 epilogue: tcgen05.ld of their 32-lane slice, C -= acc in global memory; for full tile
//           rows each thread fetches its 128 C values before the accumulator is ready.
// A second epilogue mode forms U12 = inv(L11) P A12 for the same factorisation step: A = inv(L11)
// (split, 128 x 128), B = (P A12)^T (split, written by the swap/pack kernel); the epilogue stores U12
// into the panel rows of the matrix and its transposed TF32 split over the B operand, where the
// trailing update then reads it.
// Every mbarrier wait is bounded (about 2 s of SM clock); on expiry the kernel records a status bit,
// stops issuing work, drains the copies it issued, frees its TMEM and returns. For testing that path
// (args.probe) each CTA first waits, before anything is in flight, on a barrier that nothing
// signals, with a limit of about 1 ms: the wait expires, the status bit is set and the CTA goes
// straight to its teardown.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstdio>

#include "bte_kernels.h"

namespace bte {
namespace {

#ifndef BTE_TC_BN
#define BTE_TC_BN 128
#endif
// KP: panel width (K of one panel's update); KS: K capacity of the operand workspace, the depth of
// the two-panel update
constexpr int BM = 128, BN = BTE_TC_BN, BK = 32, KP = 128, KS = 2 * KP;
static_assert(BN == 128 || BN == 256, "tile width");
// Operand stages and C staging slots share the 227 KB of shared memory (64 KB and 16 KB each).
#ifndef BTE_TC_STAGES
#define BTE_TC_STAGES 2
#endif
#ifndef BTE_TC_CSLOTS
#define BTE_TC_CSLOTS 4
#endif
constexpr int STAGES = BTE_TC_STAGES;
constexpr int A_BOX = BM * BK * 4;                // 16 KB
constexpr int B_BOX = BN * BK * 4;                // 16 or 32 KB
constexpr int STAGE_BYTES = 2 * A_BOX + 2 * B_BOX;  // A_hi, A_lo, B_hi, B_lo
#ifndef BTE_TC_CW
#define BTE_TC_CW 32
#endif
// C chunk width (columns): 32 = one 128-byte swizzle row, 16 = one 64-byte swizzle row
constexpr int CW = BTE_TC_CW;
static_assert(CW == 32 || CW == 16, "C chunk width");
constexpr int CSWZ_MASK = CW == 32 ? 7 : 3;       // 16-byte chunk index ^= (row >> CSWZ_SHIFT) & mask
constexpr int CSWZ_SHIFT = CW == 32 ? 0 : 1;
constexpr int CSLOTS = BTE_TC_CSLOTS;             // C staging slots
constexpr int CSLOT_BYTES = BM * CW * 4;          // 16 or 8 KB
constexpr int NTHREADS = 192;
constexpr long long kWaitCycles = 1ll << 32;     // ~2 s at 2 GHz
constexpr long long kProbeCycles = 1ll << 21;    // ~1 ms: the probe's wait
constexpr unsigned kTimeoutBit = 8u;

// instruction descriptor, kind::tf32 (formed per tile shape in the kernel): D = F32 (bits 4-5 = 1),
// A = B = TF32 (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at
// bits 24-28

struct Smem {
  alignas(1024) unsigned char stage[STAGES][STAGE_BYTES];
  alignas(1024) unsigned char cbuf[CSLOTS][CSLOT_BYTES];  // C chunks, 128-byte swizzled (TMA layout)
  alignas(8) uint64_t full[STAGES];
  uint64_t cfull[CSLOTS];
  uint64_t empty[STAGES];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t drain;
  uint64_t never;  // signalled by nothing: the probe's wait
  uint32_t tmem_base;
  int abort;
  int issued;    // K-chunks whose loads the producer issued
};

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// the same with cluster-scope acquire (arrivals from the other CTA of a pair)
__device__ __forceinline__ bool mbar_try_cl(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false if the phase did not complete in time or the CTA is aborting.
__device__ bool mbar_wait(Smem& s, uint64_t* b, uint32_t parity, unsigned* status, bool cl = false) {
  const long long t0 = clock64();
  while (!(cl ? mbar_try_cl(b, parity) : mbar_try(b, parity))) {
    if (*reinterpret_cast<volatile int*>(&s.abort)) return false;
    if (clock64() - t0 > kWaitCycles) {
      atomicExch(&s.abort, 1);
      atomicOr(status, kTimeoutBit);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(saddr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(saddr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(saddr(bar))
      : "memory");
}

__device__ __forceinline__ void tma_store3(const CUtensorMap* map, const void* src, int x, int y, int z) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];"
               ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(saddr(src))
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_read_all_but_last() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;                 // leading byte offset (unused for this layout)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;         // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;                 // descriptor version for tcgen05
  d |= static_cast<uint64_t>(2) << 61;                 // SWIZZLE_128B
  return d;
}

// D (+)= A B^T. CG = 1: one CTA, M = 128. CG = 2: the CTA pair of a cluster, M = 256 (each CTA
// holds 128 rows of A and half of the N rows of B at the same shared-memory offsets, and receives
// its 128 rows of D in its own tensor memory); issued by the even CTA only.
template <int CG>
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  if constexpr (CG == 1)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accum));
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n}"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

// arrive on `bar` once the MMAs issued so far have completed: in this CTA (CG = 1), or at the same
// offset in both CTAs of the pair (CG = 2)
template <int CG>
__device__ __forceinline__ void mma_commit_all(uint64_t* bar) {
  if constexpr (CG == 1)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
  else
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            saddr(bar)),
        "h"(static_cast<uint16_t>(3))
        : "memory");
}

// arrive on `bar` of this CTA only
template <int CG>
__device__ __forceinline__ void mma_commit_own(uint64_t* bar) {
  if constexpr (CG == 1)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
  else
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

// shared::cluster address of the object at p's offset in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr(p)), "r"(rank));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}

// tile load into this CTA's shared memory whose completion is counted on the pair leader's barrier
__device__ __forceinline__ void tma_load_pair(void* dst, const CUtensorMap* map, int x, int y, uint32_t cluster_bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(saddr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(cluster_bar)
      : "memory");
}


__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct TcArgs {
  float* fac;        // per-point matrices, n x n row-major
  int n;
  int row0, col0;    // origin of C inside each point's matrix
  int M, N;          // extent of C
  int tiles_m, tiles_n, total;
  int rows_a, rows_b;  // rows per point of the A and B operand arrays
  int nchunk;        // K / 32: 4 for one panel's update, 8 for a two-panel update
  int nchunk_m0;     // K / 32 for the first row tile (the two-panel inv(L11) is zero right of 128)
  int mode;          // 0: C -= A B^T;  1: C = A B^T and (bt_hi, bt_lo)[point][col][row] = split(C)
  float* bt_hi;
  float* bt_lo;
  unsigned* status;
  int probe;         // nonzero: the probe's expiring wait before any work (testing)
};

// CG = 1: one CTA per 128 x BN output tile. CG = 2: a cluster of two CTAs per 256 x 256 tile (each
// CTA stages 128 rows of A and 128 of the 256 rows of B, the even CTA issues M = 256, N = 256 MMAs
// over both CTAs' stages, each CTA's epilogue takes its 128 rows): twice the MMA work per staged
// byte of the one-CTA tile.
template <int CG>
__global__ void __launch_bounds__(NTHREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                   const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo,
                   const __grid_constant__ CUtensorMap mC, const TcArgs args) {
  static_assert(CG == 1 || (CG == 2 && BN == 128), "a CTA pair stages 128 rows of B per CTA");
  constexpr int TN = CG * BN, TM = CG * BM;  // output tile of the CTA (pair)
  constexpr int NCC = TN / CW;               // C chunks per CTA and tile
  constexpr uint32_t TCOLS = 2 * TN;         // two accumulators
  constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                             ((uint32_t)(TM >> 4) << 24);
  const int total = args.total;
  unsigned* status = args.status;
  extern __shared__ unsigned char raw[];
  Smem& s = *reinterpret_cast<Smem*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = CG == 2 ? static_cast<int>(blockIdx.x & 1) : 0;  // CTA within the pair
  const int cid = blockIdx.x / CG, ncl = gridDim.x / CG;            // tile scheduler unit

  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) mbar_init(&s.full[i], 1), mbar_init(&s.empty[i], 1);
    for (int i = 0; i < 2; ++i) mbar_init(&s.tfull[i], 1), mbar_init(&s.tempty[i], 4 * CG);
    for (int i = 0; i < CSLOTS; ++i) mbar_init(&s.cfull[i], 1);
    mbar_init(&s.drain, 1);
    mbar_init(&s.never, 1);
    s.abort = 0;
    s.issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    if constexpr (CG == 1) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&s.tmem_base)),
                   "r"(TCOLS));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    } else {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&s.tmem_base)),
                   "r"(TCOLS));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  if constexpr (CG == 2) cluster_sync();  // both CTAs' barriers exist before any cross-CTA signal
  else __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s.tmem_base;
  const int per_point = args.tiles_m * args.tiles_n;
  if (args.probe) {
    // nothing is in flight yet: the wait expires, and every role below sees the abort and skips
    // its work
    if (threadIdx.x == 0) {
      const long long t0 = clock64();
      while (!mbar_try(&s.never, 0)) {
        if (clock64() - t0 > kProbeCycles) {
          s.abort = 1;
          atomicOr(status, kTimeoutBit);
          break;
        }
      }
    }
    __syncwarp();
    if constexpr (CG == 2) cluster_sync();
    else __syncthreads();
  }
  const bool run = !*reinterpret_cast<volatile int*>(&s.abort);

  if (warp == 0) {
    if (lane == 0 && run) {  // --------------------------------------------------------- producer
      int st = 0;
      uint32_t ph = 0;
      for (int t = cid; t < total; t += ncl) {
        const int p = t / per_point, r = t % per_point;
        const int ya = p * args.rows_a + (r / args.tiles_n) * TM + rank * BM;
        const int yb = p * args.rows_b + (r % args.tiles_n) * TN + rank * BN;
        const int nch = r < args.tiles_n ? args.nchunk_m0 : args.nchunk;
        bool ok = true;
        for (int c = 0; c < nch; ++c) {
          if (!mbar_wait(s, &s.empty[st], ph ^ 1u, status, CG == 2)) { ok = false; break; }
          unsigned char* d = s.stage[st];
          if constexpr (CG == 1) {
            mbar_expect_tx(&s.full[st], STAGE_BYTES);
            tma_load(d, &mAhi, c * BK, ya, &s.full[st]);
            tma_load(d + A_BOX, &mAlo, c * BK, ya, &s.full[st]);
            tma_load(d + 2 * A_BOX, &mBhi, c * BK, yb, &s.full[st]);
            tma_load(d + 2 * A_BOX + B_BOX, &mBlo, c * BK, yb, &s.full[st]);
          } else {
            // both CTAs' bytes complete on the even CTA's barrier, which expects them all
            if (rank == 0) mbar_expect_tx(&s.full[st], 2 * STAGE_BYTES);
            const uint32_t bar = cluster_addr(&s.full[st], 0);
            tma_load_pair(d, &mAhi, c * BK, ya, bar);
            tma_load_pair(d + A_BOX, &mAlo, c * BK, ya, bar);
            tma_load_pair(d + 2 * A_BOX, &mBhi, c * BK, yb, bar);
            tma_load_pair(d + 2 * A_BOX + B_BOX, &mBlo, c * BK, yb, bar);
          }
          s.issued += 1;
          if (++st == STAGES) st = 0, ph ^= 1u;
        }
        if (!ok) break;
      }
      // producer tail: every stage handed out must have been released by its MMAs
      if (!*reinterpret_cast<volatile int*>(&s.abort)) {
        for (int i = 0; i < STAGES; ++i) {
          if (!mbar_wait(s, &s.empty[st], ph ^ 1u, status, CG == 2)) break;
          if (++st == STAGES) st = 0, ph ^= 1u;
        }
      } else if (CG == 2) {
        // after an abort this CTA cannot see its own loads complete (they count on the other
        // CTA's barrier): give any still in flight time to land before the CTA exits
        const long long t0 = clock64();
        while (clock64() - t0 < (1ll << 21)) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0 && run) {  // ----------------------------------------- MMA issuer
      int st = 0, acc = 0;
      uint32_t ph = 0, aph = 0;
      int consumed = 0;
      for (int t = cid; t < total; t += ncl) {
        if (!mbar_wait(s, &s.tempty[acc], aph ^ 1u, status, CG == 2)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + acc * TN;
        const int nch = t % per_point < args.tiles_n ? args.nchunk_m0 : args.nchunk;
        bool ok = true;
        for (int c = 0; c < nch; ++c) {
          if (!mbar_wait(s, &s.full[st], ph, status, CG == 2)) { ok = false; break; }
          ++consumed;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = saddr(s.stage[st]);
          const uint32_t a1 = a0 + A_BOX, b0 = a0 + 2 * A_BOX, b1 = b0 + B_BOX;
#pragma unroll
          for (int k = 0; k < BK / 8; ++k) {
            const uint32_t off = k * 32;  // 8 tf32 = 32 bytes inside the 128-byte swizzle row
            mma_tf32<CG>(d, sdesc(a1 + off), sdesc(b0 + off), IDESC, (c | k) ? 1u : 0u);  // a_lo b_hi
            mma_tf32<CG>(d, sdesc(a0 + off), sdesc(b1 + off), IDESC, 1u);                 // a_hi b_lo
            mma_tf32<CG>(d, sdesc(a0 + off), sdesc(b0 + off), IDESC, 1u);                 // a_hi b_hi
          }
          mma_commit_all<CG>(&s.empty[st]);
          if (++st == STAGES) st = 0, ph ^= 1u;
        }
        if (!ok) break;
        mma_commit_all<CG>(&s.tfull[acc]);
        if (++acc == 2) acc = 0, aph ^= 1u;
      }
      // drain: loads issued but not consumed must land before the CTA exits
      if (*reinterpret_cast<volatile int*>(&s.abort)) {
        for (int q = consumed; q < *reinterpret_cast<volatile int*>(&s.issued); ++q) {
          const long long t0 = clock64();
          while (!mbar_try(&s.full[st], ph) && clock64() - t0 < kWaitCycles) {
          }
          if (++st == STAGES) st = 0, ph ^= 1u;
        }
      }
      // every MMA issued by this thread has retired once the drain barrier completes
      mma_commit_own<CG>(&s.drain);
      const long long t0 = clock64();
      while (!mbar_try(&s.drain, 0) && clock64() - t0 < kWaitCycles) {
      }
    }
  } else {  // ------------------------------------------------------------------------- epilogue
    // C moves through CSLOTS 16 KB shared-memory slots in 128 x 32 chunks: TMA load (mode 0), C -= acc
    // (or C = acc) by the thread owning the row (its TMEM lane), TMA store. One leader thread waits
    // on the barriers and issues the bulk copies; the four warps meet at a named barrier, so a
    // timeout seen by the leader ends every epilogue thread at the same point.
    const int sub = warp & 3;  // TMEM lane quarter this warp may access
    const int trow = sub * 32 + lane;
    const bool leader = warp == 2 && lane == 0;
    const bool load_c = args.mode == 0;
    auto cx = [&](int t, int ch) { return args.col0 + ((t % per_point) % args.tiles_n) * TN + CW * ch; };
    auto cy = [&](int t) { return args.row0 + ((t % per_point) / args.tiles_n) * TM + rank * BM; };
    auto issue_c = [&](int t, int ch, int slot) {
      mbar_expect_tx(&s.cfull[slot], CSLOT_BYTES);
      tma_load3(s.cbuf[slot], &mC, cx(t, ch), cy(t), t / per_point, &s.cfull[slot]);
    };
    // C load number q (the q-th chunk of this CTA) goes to slot q % CSLOTS, phase (q / CSLOTS) & 1
    auto chunk_at = [&](int q, int& tq, int& chq) {
      tq = cid + (q / NCC) * ncl;
      chq = q % NCC;
    };
    int c_issued = 0, c_done = 0;  // leader's count of C loads issued and waited for
    if (leader && load_c && run)
      for (int q = 0; q < CSLOTS; ++q) {
        int tq, chq;
        chunk_at(q, tq, chq);
        if (tq >= total) break;
        issue_c(tq, chq, q % CSLOTS);
        ++c_issued;
      }
    int acc = 0, g = 0;
    uint32_t aph = 0;
    bool stop = !run;
    for (int t = cid; t < total && !stop; t += ncl) {
      const int p = t / per_point, r = t % per_point;
      const int row = (r / args.tiles_n) * TM + rank * BM + trow;
      const int col0 = (r % args.tiles_n) * TN;
      if (leader && !mbar_wait(s, &s.tfull[acc], aph, status, CG == 2)) atomicExch(&s.abort, 1);
      for (int ch = 0; ch < NCC; ++ch, ++g) {
        const int slot = g % CSLOTS;
        if (leader && load_c && !*reinterpret_cast<volatile int*>(&s.abort)) {
          if (mbar_wait(s, &s.cfull[slot], (g / CSLOTS) & 1, status)) ++c_done;
          else atomicExch(&s.abort, 1);
        }
        epi_bar();
        if (*reinterpret_cast<volatile int*>(&s.abort)) {
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t v[32];
        if constexpr (CW == 32) tmem_ld32(tmem + acc * TN + ch * CW + ((sub * 32) << 16), v);
        else tmem_ld16(tmem + acc * TN + ch * CW + ((sub * 32) << 16), v);
        float4* cs = reinterpret_cast<float4*>(s.cbuf[slot] + trow * (CW * 4));
#pragma unroll
        for (int j = 0; j < CW / 4; ++j) {
          // TMA swizzle: 16-byte chunk index ^ row bits (128-byte rows: row % 8; 64-byte: (row / 2) % 4)
          float4* q = cs + (j ^ ((trow >> CSWZ_SHIFT) & CSWZ_MASK));
          float4 x;
          if (load_c) {
            x = *q;
            x.x -= __uint_as_float(v[4 * j]);
            x.y -= __uint_as_float(v[4 * j + 1]);
            x.z -= __uint_as_float(v[4 * j + 2]);
            x.w -= __uint_as_float(v[4 * j + 3]);
          } else {
            x = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]), __uint_as_float(v[4 * j + 2]),
                            __uint_as_float(v[4 * j + 3]));
          }
          *q = x;
        }
        if (!load_c && row < args.M) {
          // transposed split of U12: lanes are consecutive rows, so each column's store is coalesced
          const int c0 = col0 + ch * CW;
          float* bh = args.bt_hi + static_cast<size_t>(p) * args.rows_b * KS + row;
          float* bl = args.bt_lo + static_cast<size_t>(p) * args.rows_b * KS + row;
#pragma unroll
          for (int j = 0; j < CW; ++j) {
            if (c0 + j >= args.N) break;
            uint32_t h;
            const float x = __uint_as_float(v[j]);
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
            bh[static_cast<size_t>(c0 + j) * KS] = __uint_as_float(h);
            bl[static_cast<size_t>(c0 + j) * KS] = x - __uint_as_float(h);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        epi_bar();
        if (leader) {
          // store this chunk; wait only until the previous chunk's store has read its slot, then
          // refill that slot (the store just issued overlaps the next chunk)
          tma_store3(&mC, s.cbuf[slot], cx(t, ch), cy(t), p);
          bulk_wait_read_all_but_last();
          if (load_c && g >= 1) {
            int t2, ch2;
            chunk_at(g - 1 + CSLOTS, t2, ch2);
            if (t2 < total) issue_c(t2, ch2, (g - 1) % CSLOTS), ++c_issued;
          }
        }
      }
      if (stop) break;
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        // the accumulator is free again (for a pair: counted on the even CTA, whose MMAs write it)
        if constexpr (CG == 1) mbar_arrive(&s.tempty[acc]);
        else mbar_arrive_remote(cluster_addr(&s.tempty[acc], 0));
      }
      if (++acc == 2) acc = 0, aph ^= 1u;
    }
    if (leader) {
      bulk_wait_all();
      // loads issued but not waited for (only after an abort) must land before the CTA exits
      for (int q = c_done; q < c_issued; ++q) {
        const long long t0 = clock64();
        while (!mbar_try(&s.cfull[q % CSLOTS], (q / CSLOTS) & 1) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
  }

  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  // a pair's MMAs write both CTAs' tensor memory and signal both CTAs' barriers: neither CTA frees
  // its tensor memory or exits before the other is done
  if constexpr (CG == 2) cluster_sync();
  else __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if constexpr (CG == 1)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
    else
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2-D K-major operand array of `rows` rows of `kext` floats, boxes of box_rows x 32, 128-byte swizzle
bool make_map(CUtensorMap* m, float* base, size_t rows, int box_rows, int kext) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(kext), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(kext) * 4};
  cuuint32_t box[2] = {BK, static_cast<cuuint32_t>(box_rows)};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The per-point matrices as a 3-D tensor [point][row][col] (so tiles are clipped at each point's
// edge), boxes of 128 rows x 32 columns, 128-byte swizzle: the epilogue's C chunks.
bool make_cmap(CUtensorMap* m, float* fac, int nx, int n) {
  auto enc = get_encode();
  if (!enc || (n & 3) != 0) return false;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(n), static_cast<cuuint64_t>(n), static_cast<cuuint64_t>(nx)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(n) * 4, static_cast<cuuint64_t>(n) * n * 4};
  cuuint32_t box[3] = {CW, BM, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, fac, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CW == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// tensor maps of the workspace parts (tc_ws_part numbering) and of the matrices (C)
enum { kMapC = 10 };
struct Maps {
  void* ws = nullptr;
  float* fac = nullptr;
  int nx = 0, n = 0;
  CUtensorMap m[11];
  bool ok = false;
};

Maps& maps_for(float* fac, void* ws, int nx, int n) {
  static Maps maps;
  if (!maps.ok || maps.ws != ws || maps.fac != fac || maps.nx != nx || maps.n != n) {
    const size_t rows = static_cast<size_t>(nx) * (n - KP);
    maps.ok = true;
    // L21 split (A of the updates, boxes of BM rows); (P A12)^T and U12^T splits (B, boxes of BN rows)
    for (int part : {0, 1, 2, 3, 6, 7})
      maps.ok = maps.ok && make_map(&maps.m[part], tc_ws_part(ws, nx, n, part), rows, part < 2 ? BM : BN, KS);
    // inv(L11) of one panel and of a two-panel block (A of the U12 products)
    for (int part : {4, 5})
      maps.ok = maps.ok && make_map(&maps.m[part], tc_ws_part(ws, nx, n, part), static_cast<size_t>(nx) * KP, BM, KP);
    for (int part : {8, 9})
      maps.ok = maps.ok && make_map(&maps.m[part], tc_ws_part(ws, nx, n, part), static_cast<size_t>(nx) * KS, BM, KS);
    maps.ok = maps.ok && make_cmap(&maps.m[kMapC], fac, nx, n);
    maps.ws = ws;
    maps.fac = fac;
    maps.nx = nx;
    maps.n = n;
    cudaFuncSetAttribute(tc_gemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(sizeof(Smem) + 1024));
    cudaFuncSetAttribute(tc_gemm_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(sizeof(Smem) + 1024));
  }
  return maps;
}

int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  return sms;
}

void launch(const Maps& mp, int ia, int ib, const TcArgs& a, cudaStream_t st) {
  const int grid = a.total < sm_count() ? a.total : sm_count();
  tc_gemm_kernel<1><<<grid, NTHREADS, sizeof(Smem) + 1024, st>>>(mp.m[ia], mp.m[ia + 1], mp.m[ib], mp.m[ib + 1],
                                                                mp.m[kMapC], a);
}

cudaLaunchConfig_t pair_config(int clusters, cudaStream_t st, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t c{};
  c.gridDim = dim3(2 * clusters);
  c.blockDim = dim3(NTHREADS);
  c.dynamicSmemBytes = sizeof(Smem) + 1024;
  c.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  c.attrs = attr;
  c.numAttrs = 1;
  return c;
}

// CTA pairs that can be resident at once (0: the pair kernel is not available)
int pair_clusters() {
  static int n = -1;
  if (n < 0) {
    n = 0;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t c = pair_config(sm_count() / 2, nullptr, attr);
    int k = 0;
    if (cudaFuncSetAttribute(tc_gemm_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sizeof(Smem) + 1024)) == cudaSuccess &&
        cudaOccupancyMaxActiveClusters(&k, tc_gemm_kernel<2>, &c) == cudaSuccess)
      n = k;
    cudaGetLastError();
  }
  return n;
}

// C -= A B^T over 256 x 256 tiles, one CTA pair per tile (mode 0 only)
void launch_pair(const Maps& mp, const TcArgs& a, cudaStream_t st) {
  const int clusters = a.total < pair_clusters() ? a.total : pair_clusters();
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t c = pair_config(clusters, st, attr);
  cudaLaunchKernelEx(&c, tc_gemm_kernel<2>, mp.m[0], mp.m[1], mp.m[6], mp.m[7], mp.m[kMapC], a);
}

// C -= A B^T over the block of C at (row0, col0) of every point: A = L21 split (parts 0, 1), B =
// U12^T split (parts 6, 7), depth nchunk * 32
void gemm(Maps& mp, float* fac, int nx, int n, int row0, int col0, int M, int N, int nchunk, unsigned* status,
          cudaStream_t st, int probe) {
  if (M <= 0 || N <= 0 || !mp.ok) return;
  TcArgs a{};
  a.fac = fac;
  a.n = n;
  a.row0 = row0;
  a.col0 = col0;
  a.M = M;
  a.N = N;
  a.tiles_m = (M + BM - 1) / BM;
  a.tiles_n = (N + BN - 1) / BN;
  a.total = nx * a.tiles_m * a.tiles_n;
  a.rows_a = a.rows_b = n - KP;
  a.nchunk = a.nchunk_m0 = nchunk;
  a.mode = 0;
  a.status = status;
  a.probe = probe;
  launch(mp, 0, 6, a, st);
}

// U12 = inv(L11) (P A12) for the M = 128 or 256 panel rows at row0 and the N columns at col0; A =
// the inverse split (parts 4, 5 or 8, 9), B = (P A12)^T split (parts 2, 3); U12 goes into the matrix
// and, transposed and split, into parts 6, 7
void u12(Maps& mp, float* fac, void* ws, int nx, int n, int row0, int col0, int M, int N, unsigned* status,
         cudaStream_t st, int probe) {
  if (N <= 0 || !mp.ok) return;
  TcArgs a{};
  a.fac = fac;
  a.n = n;
  a.row0 = row0;
  a.col0 = col0;
  a.M = M;
  a.N = N;
  a.tiles_m = M / BM;
  a.tiles_n = (N + BN - 1) / BN;
  a.total = nx * a.tiles_m * a.tiles_n;
  a.rows_a = M;
  a.rows_b = n - KP;
  a.nchunk = M / BK;
  a.nchunk_m0 = KP / BK;  // the first 128 rows of a two-panel inverse are zero beyond column 128
  a.mode = 1;
  a.bt_hi = tc_ws_part(ws, nx, n, 6);
  a.bt_lo = tc_ws_part(ws, nx, n, 7);
  a.status = status;
  a.probe = probe;
  launch(mp, M == KP ? 4 : 8, 2, a, st);
}

}  // namespace

// Workspace, floats: parts 0-3 and 6-7 are [nx][n - 128][256] (L21 split, (P A12)^T split, U12^T
// split), parts 4-5 [nx][128][128] (one panel's inv(L11) split), parts 8-9 [nx][256][256] (a
// two-panel block's inv(L11) split).
size_t tc_workspace_bytes(int nx, int n, int nbmax) {
  if (nbmax != KP || n <= KP || (n & 3) != 0) return 0;
  return (6ull * nx * static_cast<size_t>(n - KP) * KS + 2ull * nx * KP * KP + 2ull * nx * KS * KS) * sizeof(float);
}

float* tc_ws_part(void* ws, int nx, int n, int part) {
  if (!ws) return nullptr;
  const size_t big = static_cast<size_t>(nx) * (n - KP) * KS, small = static_cast<size_t>(nx) * KP * KP;
  const size_t two = static_cast<size_t>(nx) * KS * KS;
  float* f = static_cast<float*>(ws);
  if (part < 4) return f + part * big;
  if (part < 6) return f + 4 * big + (part - 4) * small;
  if (part < 8) return f + 4 * big + 2 * small + (part - 6) * big;
  return f + 6 * big + 2 * small + (part - 8) * two;
}

bool tc_matrix_map(void* map, float* fac, int nx, int n) {
  static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
  return CW == 32 && make_cmap(static_cast<CUtensorMap*>(map), fac, nx, n);
}

bool tc_available() {
  int dev = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return false;
  if (p.major != 10) return false;
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, tc_gemm_kernel<1>) != cudaSuccess) return false;
  return get_encode() != nullptr;
}

void tc_lu_gemm(float* fac, int nx, int n, int k0, int ncols, void* ws, unsigned* status, cudaStream_t st,
                int probe) {
  Maps& mp = maps_for(fac, ws, nx, n);
  gemm(mp, fac, nx, n, k0 + KP, k0 + KP, n - k0 - KP, ncols, KP / BK, status, st, probe);
}

void tc_lu_u12(float* fac, int nx, int n, int k0, int ncols, void* ws, unsigned* status, cudaStream_t st,
               int probe) {
  Maps& mp = maps_for(fac, ws, nx, n);
  u12(mp, fac, ws, nx, n, k0, k0 + KP, KP, ncols, status, st, probe);
}

void tc_lu_u12_pair(float* fac, int nx, int n, int k0, void* ws, unsigned* status, cudaStream_t st, int probe) {
  Maps& mp = maps_for(fac, ws, nx, n);
  u12(mp, fac, ws, nx, n, k0, k0 + KS, KS, n - k0 - KS, status, st, probe);
}

void tc_lu_gemm_pair(float* fac, int nx, int n, int k0, void* ws, unsigned* status, cudaStream_t st, int probe,
                     int cg) {
  Maps& mp = maps_for(fac, ws, nx, n);
  const int M = n - k0 - KS;
  if (M <= 0 || !mp.ok) return;
  if (cg == 1 || pair_clusters() < 1) {
    gemm(mp, fac, nx, n, k0 + KS, k0 + KS, M, M, KS / BK, status, st, probe);
    return;
  }
  TcArgs a{};
  a.fac = fac;
  a.n = n;
  a.row0 = a.col0 = k0 + KS;
  a.M = a.N = M;
  a.tiles_m = a.tiles_n = (M + 2 * BM - 1) / (2 * BM);
  a.total = nx * a.tiles_m * a.tiles_n;
  a.rows_a = a.rows_b = n - KP;
  a.nchunk = a.nchunk_m0 = KS / BK;
  a.mode = 0;
  a.status = status;
  a.probe = probe;
  launch_pair(mp, a, st);
}

}  // namespace bte
