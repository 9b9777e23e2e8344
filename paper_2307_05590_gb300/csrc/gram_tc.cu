// Tall complex64 Gram products on the fifth-generation tensor cores (the mixed-precision
// projection of Eqs. (17)-(19): K_r = U^H (K U), C_r = U^H C U, eps M_r, b = U^H C O, all of the
// form G = A^H diag(w) B over the N rows of the full-order space).
//
// A complex product is four real ones: with A = Ar + i Ai and B' = diag(w) B = Br + i Bi,
//   Re G = Ar^T Br + Ai^T Bi,   Im G = Ar^T Bi - Ai^T Br,
// so one real GEMM of [Ar Ai]^T (2 ma x rows) by [Br Bi] (rows x 2 mb) gives all four blocks.
// Each real operand is split into two parts, x = x_hi + x_lo (x_hi = tf32(x) rounded, x_lo =
// x - x_hi exactly, of which the MMA reads the TF32 part), and a_hi b_hi + a_hi b_lo + a_lo b_hi
// is accumulated in FP32 in tensor memory (three tcgen05.mma of kind::tf32 per product tile):
// products accurate to about 2^-20 instead of TF32's 1e-3.  The rows are the reduction
// dimension (K of the MMA).
//
// Per CTA (one per SM, 16 warps, a contiguous range of rows): chunks of 16 rows of A, B and w are copied
// into shared memory by the bulk-copy engine (cp.async.bulk, completion on an mbarrier), two raw
// stages in flight; all threads convert a raw chunk into the K-major operand tiles (real and
// imaginary rows, hi and lo parts; two operand stages), one thread issues the MMAs and commits
// them to the stage's mbarrier, which releases the operand stage for the chunk after next.  The
// accumulator (Mpad x Npad FP32, Mpad = 128 per M tile) lives in tensor memory; after every 8
// chunks (128 rows) the CTA waits for its MMAs, reads the accumulator with tcgen05.ld and adds it
// into its float64 partial block (the tensor cores' FP32 accumulation then spans 128 rows only),
// and a second kernel sums the blocks over the CTAs in float64 in a fixed order and maps them to
// the complex G.
//
// Operand tiles in shared memory: no swizzle, K-major core matrices of 8 rows x 16 bytes (4
// TF32 values); within a tile of K = 16 the four core matrices of an 8-row group are adjacent
// (leading byte offset 128: next core matrix along K), and 8-row groups follow each other every
// 512 bytes (stride byte offset).  The MMA's K step of 8 starts 256 bytes further.
//
// Every wait on an mbarrier is bounded: a wait that gives up sets kStatusTimeout, the CTA waits
// (bounded) for its own copies and MMAs in flight, frees its tensor memory and returns.
#include "mrom_internal.h"

#include <algorithm>

namespace mrom {
namespace {

constexpr int kTT = 512;           // threads per CTA (16 warps)
constexpr int kMaxHalf = 112;      // ma, mb <= 112, so 2 ma, 2 mb <= 224
constexpr long long kSpinLimit = 1LL << 26;  // try_wait polls before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}


// Bounded wait for the phase with the given parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16), completing
// `bytes` of the mbarrier's transaction count.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// Shared-memory matrix descriptor of a K-major operand without swizzle (see the file comment):
// leading byte offset 128 (next core matrix along K), stride byte offset sbo (next 8-row group).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t sbo) {
  constexpr uint64_t kLbo = 128;
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((kLbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture
  return d;                // base offset 0, layout: no swizzle
}

// Instruction descriptor: kind::tf32, FP32 accumulator, A and B K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
  return (1u << 4)                       // D format: F32
         | (2u << 7)                     // A format: TF32
         | (2u << 10)                    // B format: TF32
         | ((uint32_t)(n >> 3) << 17)    // N / 8
         | ((uint32_t)(m >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 8 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}

struct TcGramArgs {
  const float2* A;   // n x ma, row-major
  const float2* B;   // n x mb, row-major (unused when same_ab)
  const float* w;    // n weights of B's rows, or null
  int64_t n;
  int ma, mb, mpad, npad, same_ab, nraw;  // nraw: raw stages (bulk copies in flight), 2 or 3
  int64_t rows_per_cta;
  double* part;      // [gridDim.x][mpad][npad]
  int* status;
};

constexpr int kMaxRaw = 3;  // raw stages at most

// byte offset of element (row, k) in a K-major operand tile of K = KT (see the file comment:
// core matrices of 8 rows x 4 k, KT / 4 of them side by side per 8-row group)
template <int KT>
__device__ __forceinline__ uint32_t op_off(int row, int k) {
  return (uint32_t)((row >> 3) * (32 * KT) + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// KT rows (the MMA's K) per chunk; g.nraw chunks' bulk copies in flight, two operand stages.
// NB > 0 (one M tile, npad <= 32 NB): each thread keeps its share of the partial block in
// registers (NB blocks of 8 columns, compensated float32 pairs) and stores it once at the end;
// NB = 0: the float64 partial block is accumulated in global memory at every flush.
template <int KT, int NB>
__global__ void __launch_bounds__(kTT, 1) gram_tc_kernel(const TcGramArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int kFlush = 128 / KT;  // chunks per FP32 accumulation segment (128 rows)
  constexpr int kKG = KT / 4;       // core matrices along K per 8-row group
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ma = g.ma, mb = g.mb, mpad = g.mpad, npad = g.npad, NR = g.nraw;
  const int mtiles = mpad / 128;
  // ---- shared memory carve-up
  uint64_t* raw_full = reinterpret_cast<uint64_t*>(smem);       // kMaxRaw barriers
  uint64_t* op_free = raw_full + kMaxRaw;                        // 2 barriers
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 64);
  const uint32_t a_raw_b = 8u * KT * ma, b_raw_b = g.same_ab ? 0u : 8u * KT * mb, w_raw_b = 4u * KT;
  const uint32_t raw_stage_b = (a_raw_b + b_raw_b + w_raw_b + 127u) & ~127u;
  unsigned char* raw0 = smem + 128;
  const uint32_t a_op_b = 4u * KT * mpad, b_op_b = 4u * KT * npad;
  const uint32_t op_stage_b = 2u * a_op_b + 2u * b_op_b;
  unsigned char* op0 = raw0 + NR * raw_stage_b;
  auto raw_a = [&](int s) { return reinterpret_cast<float2*>(raw0 + s * raw_stage_b); };
  auto raw_b = [&](int s) { return reinterpret_cast<float2*>(raw0 + s * raw_stage_b + a_raw_b); };
  auto raw_w = [&](int s) { return reinterpret_cast<float*>(raw0 + s * raw_stage_b + a_raw_b + b_raw_b); };
  auto a_hi = [&](int s) { return op0 + s * op_stage_b; };
  auto a_lo = [&](int s) { return op0 + s * op_stage_b + a_op_b; };
  auto b_hi = [&](int s) { return op0 + s * op_stage_b + 2 * a_op_b; };
  auto b_lo = [&](int s) { return op0 + s * op_stage_b + 2 * a_op_b + b_op_b; };

  const int64_t row0 = (int64_t)blockIdx.x * g.rows_per_cta;
  const int64_t row1 = min(g.n, row0 + g.rows_per_cta);
  const int nchunks = row1 > row0 ? (int)((row1 - row0 + KT - 1) / KT) : 0;
  auto chunk_rows = [&](int c) { return (int)min((int64_t)KT, row1 - (row0 + (int64_t)c * KT)); };
  const int ncols = mtiles * npad <= 256 ? 256 : 512;

  // ---- set-up: barriers, tensor memory, zeroed operand tiles (their padding rows stay zero)
  if (tid == 0) {
    for (int k = 0; k < kMaxRaw + 2; ++k) mbar_init(raw_full + k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  for (uint32_t o = tid * 16u; o < 2u * op_stage_b; o += kTT * 16u)
    *reinterpret_cast<uint4*>(op0 + o) = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *tslot;

  // thread 0's view of the asynchronous work in flight (for the error path)
  int tma_issued = -1;     // highest chunk whose bulk copies were issued
  int mma_last = -1;       // highest chunk whose MMAs were committed
  auto issue_copy = [&](int c) {  // thread 0: bulk copies of a full chunk into raw stage c % NR
    const int s = c % NR;
    const int64_t r = row0 + (int64_t)c * KT;
    mbar_expect_tx(raw_full + s, a_raw_b + b_raw_b + (g.w ? w_raw_b : 0u));
    bulk_g2s(raw_a(s), g.A + r * ma, a_raw_b, raw_full + s);
    if (!g.same_ab) bulk_g2s(raw_b(s), g.B + r * mb, b_raw_b, raw_full + s);
    if (g.w) bulk_g2s(raw_w(s), g.w + r, w_raw_b, raw_full + s);
    tma_issued = c;
  };
  if (tid == 0) {
    for (int c = 0; c < NR && c < nchunks; ++c)
      if (chunk_rows(c) == KT) issue_copy(c);
  }

  // this CTA's partial block (float64) += (or, on the first segment, =) the accumulator; every
  // warp reads its lane quarter (warp % 4) of each M tile, the warp sets alternate 8-column
  // blocks.  With no chunk the block is set to zero without touching tensor memory.
  const int nchunks_cta = nchunks;
  // the register block as an unevaluated float32 pair hi + lo, added to by compensated (two-sum)
  // steps on the FP32 pipe: float64 adds would cost the scarce FP64 pipe 8 NB per thread and flush
  float rhi[NB > 0 ? 8 * NB : 1], rlo[NB > 0 ? 8 * NB : 1];
#pragma unroll
  for (int k = 0; k < (NB > 0 ? 8 * NB : 1); ++k) rhi[k] = rlo[k] = 0.f;
  // With NB > 0 the accumulator of segment g (kFlush chunks) lives at tensor-memory column
  // 128 (g & 1): the MMAs of segment g + 1 run into the other half while segment g is read, two
  // chunks after its last chunk, whose MMAs the wait for its operand stage has then seen complete.
  constexpr bool kDefer = NB > 0;
  auto acc_col = [](int gseg) { return kDefer ? (uint32_t)((gseg & 1) * 128) : 0u; };
  auto flush = [&](bool first, uint32_t col) {
    const int q = warp & 3, cg = warp >> 2;
    constexpr int kCG = kTT / 128;  // warp sets sharing the lane quarters
    double* out = g.part + (size_t)blockIdx.x * mpad * npad;
    if constexpr (NB > 0) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int cb = cg * 8 + b * 8 * kCG;
        if (cb < npad && nchunks_cta > 0) {
          float v[8];
          tmem_ld8(taddr + ((uint32_t)(q * 32) << 16) + col + (uint32_t)cb, v);
#pragma unroll
          for (int k = 0; k < 8; ++k) {  // two-sum of hi and v, the rounding error into lo
            const float a = rhi[b * 8 + k], sum = a + v[k], bv = sum - a;
            rlo[b * 8 + k] += (a - (sum - bv)) + (v[k] - bv);
            rhi[b * 8 + k] = sum;
          }
        }
      }
    } else {
      for (int t = 0; t < mtiles; ++t) {
        const int m = t * 128 + q * 32 + lane;
        for (int cb = cg * 8; cb < npad; cb += 8 * kCG) {
          float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          if (nchunks_cta > 0) tmem_ld8(taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(t * npad + cb), v);
          // partial block stored [column][row]: the 32 lanes of a warp write 32 consecutive rows
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            double* o = out + (size_t)(cb + k) * mpad + m;
            *o = first ? (double)v[k] : *o + (double)v[k];
          }
        }
      }
    }
  };

  // operand descriptors of the two stages (thread 0), advanced per K step and M tile by adding
  // to the 14-bit address field (shared addresses stay below 256 KB)
  uint64_t dA0[3], dA1[3], dB0[3], dB1[3];
  {
    const uint32_t sbo = 32u * KT;
    const uint32_t pa0[3] = {smem_u32(a_hi(0)), smem_u32(a_hi(0)), smem_u32(a_lo(0))};
    const uint32_t pb0[3] = {smem_u32(b_hi(0)), smem_u32(b_lo(0)), smem_u32(b_hi(0))};
    const uint32_t pa1[3] = {smem_u32(a_hi(1)), smem_u32(a_hi(1)), smem_u32(a_lo(1))};
    const uint32_t pb1[3] = {smem_u32(b_hi(1)), smem_u32(b_lo(1)), smem_u32(b_hi(1))};
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      dA0[p] = smem_desc(pa0[p], sbo);
      dB0[p] = smem_desc(pb0[p], sbo);
      dA1[p] = smem_desc(pa1[p], sbo);
      dB1[p] = smem_desc(pb1[p], sbo);
    }
  }
  const uint32_t idesc = instr_desc(128, npad);
  const int nseg = (nchunks + kFlush - 1) / kFlush;
  auto issue_mmas = [&](int cm) {  // thread 0: the MMAs of chunk cm from operand stage cm & 1
    const int sm = cm & 1;
    tc_fence_after();
    const uint32_t dcol = taddr + acc_col(cm / kFlush);
#pragma unroll
    for (int ks = 0; ks < KT / 8; ++ks)
      for (int t = 0; t < mtiles; ++t)
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const uint64_t ad = (sm ? dA1[p] : dA0[p]) + (uint64_t)((ks * 256u + (uint32_t)t * 512u * KT) >> 4);
          const uint64_t bd = (sm ? dB1[p] : dB0[p]) + (uint64_t)((ks * 256u) >> 4);
          mma_tf32(dcol + (uint32_t)(t * npad), ad, bd, idesc, (cm % kFlush > 0 || ks > 0 || p > 0) ? 1u : 0u);
        }
    mma_commit(op_free + sm);
    mma_last = cm;
  };
  int flushed = 0;  // segments added into the float64 block so far (deferred mode)

  bool failed = false;
  int c = 0;
  for (; c < nchunks; ++c) {
    const int s = c & 1, sr = c % NR;
    const uint32_t raw_par = (uint32_t)((c / NR) & 1);
    const int rows = chunk_rows(c);
    const bool full = rows == KT;
    // the deferred flush of the previous segment: chunk c - 2 ended it, and its MMAs are complete
    // once the wait below for operand stage s has returned
    const bool dflush = kDefer && c % kFlush == 1 && c / kFlush >= 1 && flushed == c / kFlush - 1;
    // thread 0 polls (bounded); after the barrier every other thread observes the completed
    // phases with one try_wait each, which makes the copied bytes visible to it
    bool ok = true;
    if (tid == 0) {
      if (full) ok = mbar_wait(raw_full + sr, raw_par);
      if (c >= 2 && ok) ok = mbar_wait(op_free + s, (uint32_t)(((c - 2) >> 1) & 1));
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    if (tid != 0 && full) mbar_wait(raw_full + sr, raw_par);
    if (dflush) {
      if (tid != 0) mbar_wait(op_free + s, (uint32_t)(((c - 2) >> 1) & 1));  // completed: returns at once
      tc_fence_after();
      flush(false, acc_col(flushed));
      tc_fence_before();
      ++flushed;
    }
    // ---- convert chunk c into the operand tiles of stage s: one item per (complex column,
    // quad of 4 rows k), A's items first, then B's; an item reads 4 raw values (lanes along the
    // columns: conflict-free) and stores the hi and lo parts of its real and imaginary rows as
    // 16-byte vectors (4 consecutive k of one core-matrix row); two items per thread and pass,
    // their loads first
    const int64_t r0 = row0 + (int64_t)c * KT;
    const float2* ra = raw_a(sr);
    const float2* rb = g.same_ab ? ra : raw_b(sr);
    const float* rw = raw_w(sr);
    unsigned char *ah = a_hi(s), *al = a_lo(s), *bh = b_hi(s), *bl = b_lo(s);
    const int na = ma * kKG, nitems = na + mb * kKG;
    auto load_item = [&](int it, float (&x)[4], float (&y)[4]) {
      const bool isA = it < na;
      const int jt = isA ? it : it - na;
      const int mc = isA ? ma : mb;
      const int m = jt % mc, k0 = 4 * (jt / mc);
      const float2* src = isA ? ra : rb;
      const float2* gsrc = (isA || g.same_ab) ? g.A : g.B;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int kk = k0 + j;
        float2 v = make_float2(0.f, 0.f);
        float wt = 1.f;
        if (full) {
          v = src[kk * mc + m];
          if (!isA && g.w) wt = rw[kk];
        } else if (kk < rows) {
          v = gsrc[(r0 + kk) * mc + m];
          if (!isA && g.w) wt = g.w[r0 + kk];
        }
        x[j] = wt * v.x;
        y[j] = wt * v.y;
      }
    };
    auto store_item = [&](int it, const float (&x)[4], const float (&y)[4]) {
      const bool isA = it < na;
      const int jt = isA ? it : it - na;
      const int mc = isA ? ma : mb;
      const int m = jt % mc, k0 = 4 * (jt / mc);
      uint32_t hre[4], lre[4], him[4], lim[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        hre[j] = to_tf32(x[j]);  // hi: rounded to TF32; lo: the exact remainder (the MMA reads
        him[j] = to_tf32(y[j]);  // its TF32 part)
        lre[j] = __float_as_uint(x[j] - __uint_as_float(hre[j]));
        lim[j] = __float_as_uint(y[j] - __uint_as_float(him[j]));
      }
      unsigned char* hi = isA ? ah : bh;
      unsigned char* lo = isA ? al : bl;
      const uint32_t ore = op_off<KT>(m, k0), oim = op_off<KT>(mc + m, k0);
      *reinterpret_cast<uint4*>(hi + ore) = make_uint4(hre[0], hre[1], hre[2], hre[3]);
      *reinterpret_cast<uint4*>(lo + ore) = make_uint4(lre[0], lre[1], lre[2], lre[3]);
      *reinterpret_cast<uint4*>(hi + oim) = make_uint4(him[0], him[1], him[2], him[3]);
      *reinterpret_cast<uint4*>(lo + oim) = make_uint4(lim[0], lim[1], lim[2], lim[3]);
    };
    // warp 0: thread 0 issues the copies into the raw stage chunk c - 1 freed and the MMAs of
    // chunk c - 1 (converted in the previous pass) while warps 1.. convert chunk c
    if (warp == 0) {
      if (tid == 0 && c >= 1) {
        if (c - 1 + NR < nchunks && chunk_rows(c - 1 + NR) == KT) issue_copy(c - 1 + NR);
        issue_mmas(c - 1);
      }
    } else {
      constexpr int kConv = kTT - 32;  // converting threads
      for (int it = tid - 32; it < nitems; it += 2 * kConv) {
        float x0[4], y0[4], x1[4], y1[4];
        const bool two = it + kConv < nitems;
        load_item(it, x0, y0);
        if (two) load_item(it + kConv, x1, y1);
        store_item(it, x0, y0);
        if (two) store_item(it + kConv, x1, y1);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();  // raw stage sr consumed, operand stage s written
    // ---- chunk c - 1 ended a segment (float64 block in global memory): wait for its MMAs and add
    // the FP32 accumulator into this CTA's partial block before the next segment's first MMAs
    if (!kDefer && c >= 1 && (c - 1) % kFlush == kFlush - 1) {
      const int cm = c - 1;
      const bool ok = tid == 0 ? mbar_wait(op_free + (cm & 1), (uint32_t)((cm >> 1) & 1)) : true;
      if (__syncthreads_or(!ok)) {
        failed = true;
        ++c;  // chunk c was consumed
        break;
      }
      if (tid != 0) mbar_wait(op_free + (cm & 1), (uint32_t)((cm >> 1) & 1));  // completed: returns at once
      tc_fence_after();
      flush(cm < kFlush, 0u);
      tc_fence_before();
      __syncthreads();
    }
  }
  // the last chunk's MMAs, then the segments not yet added, once every MMA is complete
  if (!failed && nchunks > 0) {
    if (tid == 0) issue_mmas(nchunks - 1);
    const int last = nchunks - 1;  // (every thread knows it; mma_last is thread 0's)
    const uint32_t par = (uint32_t)((last >> 1) & 1);
    const bool ok = tid == 0 ? mbar_wait(op_free + (last & 1), par) : true;
    if (__syncthreads_or(!ok)) {
      failed = true;
    } else {
      if (tid != 0) mbar_wait(op_free + (last & 1), par);  // completed: returns at once
      tc_fence_after();
      if constexpr (kDefer) {
        for (; flushed < nseg; ++flushed) flush(false, acc_col(flushed));
      } else {
        flush(last < kFlush, 0u);  // the last segment
      }
      tc_fence_before();
      __syncthreads();
    }
  }
  if (!failed && nchunks == 0) flush(true, 0u);  // zeros for an empty range
  if constexpr (NB > 0) {  // the register block, once ([column][row] as above)
    const int q = warp & 3, cg = warp >> 2;
    constexpr int kCG = kTT / 128;
    double* out = g.part + (size_t)blockIdx.x * mpad * npad;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int cb = cg * 8 + b * 8 * kCG;
      if (cb < npad) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
          out[(size_t)(cb + k) * mpad + q * 32 + lane] = (double)rhi[b * 8 + k] + (double)rlo[b * 8 + k];
      }
    }
  }
  if (failed) {
    if (tid == 0) {
      atomicOr(g.status, kStatusTimeout);
      // bounded waits for this CTA's own copies and MMAs still in flight
      for (int k = c; k <= tma_issued; ++k) mbar_wait(raw_full + (k % NR), (uint32_t)((k / NR) & 1));
      if (mma_last >= 0) mbar_wait(op_free + (mma_last & 1), (uint32_t)((mma_last >> 1) & 1));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
  }
}

// G[i][j] = sum over the CTAs of (P[i][j] + P[ma+i][mb+j]) + i (P[i][mb+j] - P[ma+i][j]), float64,
// CTAs in order; a CTA's block P is stored [column][row]
__global__ void gram_tc_reduce_kernel(const double* __restrict__ part, int nblk, int ma, int mb, int mpad, int npad,
                                      double2* __restrict__ G, int64_t ldg) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < ma * mb; idx += gridDim.x * blockDim.x) {
    const int i = idx / mb, j = idx - (idx / mb) * mb;
    double re = 0.0, im = 0.0;
    for (int b = 0; b < nblk; ++b) {
      const double* P = part + (size_t)b * mpad * npad;
      re += P[(size_t)j * mpad + i] + P[(size_t)(mb + j) * mpad + ma + i];
      im += P[(size_t)(mb + j) * mpad + i] - P[(size_t)j * mpad + ma + i];
    }
    G[(size_t)i * ldg + j] = make_double2(re, im);
  }
}

}  // namespace

// dynamic shared memory of a launch with KT rows per chunk and nraw raw stages
size_t tall_gram_tc_smem(int ma, int mb, bool same_ab, int kt, int nraw) {
  const int mpad = 128 * ((2 * ma + 127) / 128), npad = 16 * ((2 * mb + 15) / 16);
  const size_t raw_stage = ((size_t)8 * kt * ma + (same_ab ? 0 : (size_t)8 * kt * mb) + 4 * kt + 127) & ~(size_t)127;
  return 128 + nraw * raw_stage + 2 * (2 * (size_t)4 * kt * mpad + 2 * (size_t)4 * kt * npad);
}

cudaError_t tall_gram_tc(mrom_ctx* h, const float2* A, int ma, const float2* B, int mb, const float* w, int64_t n,
                         double2* G, int64_t ldg) {
  if (ma < 1 || mb < 1 || ma > kMaxHalf || mb > kMaxHalf || n < 1) return cudaErrorInvalidValue;
  const bool same = (A == B) && (ma == mb);
  const int mpad = 128 * ((2 * ma + 127) / 128), npad = 16 * ((2 * mb + 15) / 16);
  // the largest chunk and the most copies in flight that fit: 32 rows and three raw stages keep
  // enough bytes in flight per SM to cover the memory latency at the HBM rate
  int kt = 0, nraw = 0;
  size_t smem = 0;
  for (int cand = 0; cand < 4 && kt == 0; ++cand) {
    const int k = cand < 2 ? 32 : 16, nr = (cand & 1) ? 2 : 3;
    const size_t b = std::max<size_t>(tall_gram_tc_smem(ma, mb, same, k, nr), 116 * 1024);
    if (b <= h->smem_optin) {
      kt = k;
      nraw = nr;
      smem = b;  // at least 116 KB so that one CTA runs per SM (each holds up to 512 tensor-memory columns)
    }
  }
  if (kt == 0) return cudaErrorInvalidValue;
  const int64_t chunks = (n + kt - 1) / kt;
  const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>(h->num_sms, chunks));
  const int64_t per = (chunks + nblk - 1) / nblk * kt;
  DevBuf part;
  cudaError_t e = cudaMalloc(&part.p, (size_t)nblk * mpad * npad * sizeof(double));
  if (e != cudaSuccess) return e;
  TcGramArgs a{A, same ? nullptr : B, w, n, ma, mb, mpad, npad, same ? 1 : 0, nraw, per, static_cast<double*>(part.p),
               h->d_status};
  // the float64 partial block in registers when it is one M tile of at most 128 columns
  const int nb = mpad == 128 ? (npad + 31) / 32 : 0;
  auto launch = [&](auto kernel) {
    cudaError_t x = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (x == cudaSuccess) kernel<<<nblk, kTT, smem, h->stream>>>(a);
    return x;
  };
  if (kt == 32)
    e = nb == 1 ? launch(gram_tc_kernel<32, 1>) : nb == 2 ? launch(gram_tc_kernel<32, 2>)
        : nb == 3 ? launch(gram_tc_kernel<32, 3>) : nb == 4 ? launch(gram_tc_kernel<32, 4>)
                  : launch(gram_tc_kernel<32, 0>);
  else
    e = nb == 1 ? launch(gram_tc_kernel<16, 1>) : nb == 2 ? launch(gram_tc_kernel<16, 2>)
        : nb == 3 ? launch(gram_tc_kernel<16, 3>) : nb == 4 ? launch(gram_tc_kernel<16, 4>)
                  : launch(gram_tc_kernel<16, 0>);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gram_tc_reduce_kernel<<<std::max(1, std::min(1024, (ma * mb + 255) / 256)), 256, 0, h->stream>>>(
      static_cast<double*>(part.p), nblk, ma, mb, mpad, npad, G, ldg);
  e = cudaGetLastError();
  h->launches += 2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // part is freed on return
  return e;
}

}  // namespace mrom
