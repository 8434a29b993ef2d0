// Tensor-core dilated 3x3 conv for sm_103a: implicit GEMM on tcgen05 with TMEM accumulators,
// activations staged by TMA (dilated convolution, Sec. 3.2.1; heads of Sec. 3.2 fused into
// the last layer's epilogue).
//
// GEMM view of one output row segment: D[m, co] = sum_{ky,kx,ci} A[m + kx*d, ci | row ky] W[ky,kx,ci,co]
// with M = 128 pixels of one image row, N = C output channels, K = 9 taps x C input channels.
//
// Activation layout in HBM ("row-planar"): [T][H][G][W][row bytes], G = C / 16 groups of
// 16 channels; a pixel's group row is 32 bytes in BF16 and 16 bytes in FP8 e4m3.  One TMA
// box per input row (group row x (128 + 2d, rounded up to 32) pixels x G groups) lands in
// shared memory as G planes of [pixel][row bytes]:
//   * BF16: 32-byte rows written with the 32-byte swizzle, the canonical SWIZZLE_32B K-major
//     UMMA operand; one plane = one K=16 step (SBO = 256 B per 8 pixels).  The swizzle is a
//     function of the absolute shared-memory address, so the operand of tap kx is the same
//     plane started kx*d rows later, for any d.
//   * FP8: 16-byte rows, the no-swizzle K-major operand with 16-byte core-matrix rows; a K=32
//     step spans two planes (LBO = plane stride, SBO = 128 B), and a zero plane pads C=48.
// The TMA zero fill of out-of-frame pixels and rows is the "same" zero padding.
//
// Work decomposition ("row classes"): the three input rows of output row i are i-d, i, i+d,
// so rows with the same residue mod d form independent chains.  A work unit is
// (frame, 128-pixel column strip, residue phi, segment of S consecutive rows of the chain);
// each CTA takes a contiguous range of units in (frame, phi, strip, segment) order, so the
// rows and columns a unit shares with its successors are still in L2 when they load them.
// A unit's S+2 input rows stream through a ring of TMA stages, each loaded once.  Input row k'
// feeds output rows k', k'-1, k'-2 through the vertical taps ky = 0, 1, 2; those three
// contributions are ONE MMA with N = 3C (B = the three taps' weights side by side) whose
// D columns are the three rows' accumulators: output row k of a unit accumulates at TMEM
// column base0 - C*k, a window that slides down by C columns per input row.  Blocks that
// would belong to rows outside the unit are not issued (N shrinks to C or 2C at the unit's
// edges).  Every MMA accumulates: the epilogue, right after reading a row's accumulator,
// writes the layer's bias into those columns (FP8: bias / dequantisation factor), so each
// row starts from its bias.  Accumulation order inside a row is fixed (bias, then ky, kx,
// k-step ascending), so the result does not depend on scheduling, grid size or batch
// composition.
//
// Warp roles (224 threads): warps 0-3 epilogue (TMEM lane quarter = warp index), warp 4 TMA
// producer, warp 5 TMEM allocator and MMA issuer, warp 6 waiter (the MMA warp's mbarrier
// waits, handed over through named barriers).  Every mbarrier wait is bounded: on timeout
// the kernel sets *err, the producer and epilogue stop, the MMA warp finishes its row
// sequence without waiting, the MMAs and TMA loads in flight are drained (bounded), TMEM is
// freed and the kernel returns.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <mutex>
#include <type_traits>

#include "sml_internal.h"
#include "tc_ptx.cuh"

namespace sml {

namespace {

constexpr int kEpiWarps = 4;
constexpr int kThreads = 224;
constexpr int kMinStages = 4;  // the handoff protocol needs a ring of at least 2 handoff groups
constexpr int kTmemCols = 512;  // TMEM columns of a CTA that has its SM to itself
constexpr int kPairTmemCols = 256;  // of each of two CTAs sharing an SM (PAIR instances)
constexpr int kMaxSeg = 10;
constexpr int kMaxStages = 16;

// Kernel arguments; bias, dequantisation factors and head weights travel by value so the
// epilogue's FMAs read them from the constant bank.
struct TcKArgs {
  const uint8_t* bimg;
  float bias[64];
  float deq[64];
  float head_w[kMaxHeads * 64];  // [nh][C]
  float head_b[12];
  int nh;                        // heads: 5, or 9 with the uncertainty heads
  float out_inv_scale;
  uint8_t* out;
  float* maps;
  float* logits;
  int T, H, W, d;
  int NS, NQ;          // column strips, segments per residue class
  uint32_t units;      // T * NS * d * NQ
  uint32_t stage_bytes, plane_stride, tx_bytes;
  int nstages;
  // runtime-K instances (CI = 0): K steps per tap, input groups loaded per row, planes per
  // stage, bytes of the B image; output: first group and groups per pixel row of the buffer
  int nks, g_in, g_planes;
  uint32_t bimg_bytes;
  int out_g0, out_gt;
  const float* bias_dev;  // device [co] bias (BF16 training), read instead of bias[] when set
  const uint8_t* mask;    // DGRAD: the lower layer's activations, laid out like out
  // Failure-path test settings: the give-up time of the waits on other roles (kWaitLimitNs
  // unless a test shortens it) and a CTA whose producer issues no load at all (-1: none), so
  // that its consumers' waits run out with no copy of that CTA in flight
  unsigned long long wait_ns;
  int poison_cta;
  // FP8 rows loaded as 32-byte pixel pairs (frames of even width): the box starts at pixel
  // j0 - d - pair_off (pair_off = d & 1 keeps the start even) and the A operand pair_off
  // pixels into the box; -1: one 16-byte row per pixel
  int pair_off;
  int* err;
};

// Compile-time shape of one layer: CI input channels (K = 9 taps x CI), CO output channels
// (N = 3 CO per MMA).  CI = 0 is the runtime-K instance: the K-dependent sizes come from the
// kernel arguments instead (dense-block layers, whose CI grows along the block).
// PAIR: two CTAs share each SM, each with half of its TMEM and shared memory, so that two MMA
// issue streams feed one tensor pipe (one CTA's MMA warp leaves the pipe idle while it
// commits, hands over and keeps its books; measured in FP8 layers and last layers: see the
// launcher).
template <int CI, int CO, int PREC, bool PAIR = false>
struct TcCfg {
  static constexpr int G = CI / 16;                       // 16-channel input groups stored in HBM
  static constexpr int GO = CO / 16;                      // output groups
  static constexpr int KSTEP = PREC == kBF16 ? 16 : 32;   // K per MMA instruction
  static constexpr int NKS = (CI + KSTEP - 1) / KSTEP;    // MMAs per tap
  static constexpr int GP = PREC == kBF16 ? G : 2 * NKS;  // planes in shared memory (FP8: zero pad)
  static constexpr int BBLK = 3 * (CO / 8) * 256;         // bytes of one (kx, k-step) B block: N = 3 CO
  static constexpr int BIMG = 3 * NKS * BBLK;
  // S = output rows per unit.  Output row k accumulates at columns BASE0 - CO*k .. + CO, and an
  // input row's MMA only writes the columns of the unit's rows it feeds, so a unit spans
  // columns [BASE0 - CO*(S-1), BASE0 + CO).  With the whole TMEM: BASE0 = (S+1) CO, i.e.
  // [2 CO, (S+2) CO), S <= 512/CO - 2; with half of it (PAIR): BASE0 = (S-1) CO, i.e.
  // [0, S CO), S <= 256/CO.
  static constexpr int TMEM_COLS = PAIR ? kPairTmemCols : kTmemCols;
  static constexpr int SEG_FIT = PAIR ? kPairTmemCols / CO : kTmemCols / CO - 2;
  static constexpr int SEG = SEG_FIT < kMaxSeg ? SEG_FIT : kMaxSeg;
  static constexpr uint32_t BASE0 = (uint32_t)(PAIR ? SEG - 1 : SEG + 1) * CO;  // TMEM column of output row 0
  static_assert(BASE0 + CO <= (uint32_t)TMEM_COLS && BASE0 >= (uint32_t)(CO * (SEG - 1)),
                "a unit's accumulators fit the CTA's TMEM columns");
  static constexpr uint32_t IDESC1 = instr_desc(PREC, kTileM, CO);
  static constexpr uint32_t IDESC2 = instr_desc(PREC, kTileM, 2 * CO);
  static constexpr uint32_t IDESC3 = instr_desc(PREC, kTileM, 3 * CO);
};

// Unit -> (t, phi, strip, q), q fastest: consecutive units are the next segment of the same
// row chain (sharing two input rows) and then the neighbouring strip (sharing halo columns),
// so with contiguous unit ranges per CTA those re-reads hit L2.  Every role walks its CTA's
// range with a cursor: the first unit is decoded with divisions, each later one by a carry
// chain, and the residue class's row count is recomputed only when phi changes (measured: the
// divisions of a full decode cost the issuing warp about 500 cycles per unit).  32-bit
// arithmetic (unit counts stay far below 2^31).
struct UnitCursor {
  int t, phi, s, q, n_class;
  __device__ __forceinline__ void set_class(const TcKArgs& a) { n_class = phi < a.H ? (a.H - phi + a.d - 1) / a.d : 0; }
  __device__ __forceinline__ void init(const TcKArgs& a, uint32_t u) {
    const uint32_t nq = (uint32_t)a.NQ, d = (uint32_t)a.d, ns = (uint32_t)a.NS;
    const uint32_t r = u / nq;
    q = (int)(u - r * nq);
    const uint32_t r2 = r / ns;
    s = (int)(r - r2 * ns);
    const uint32_t r3 = r2 / d;
    phi = (int)(r2 - r3 * d);
    t = (int)r3;
    set_class(a);
  }
  __device__ __forceinline__ void next(const TcKArgs& a) {
    if (++q < a.NQ) return;
    q = 0;
    if (++s < a.NS) return;
    s = 0;
    if (++phi == a.d) {
      phi = 0;
      ++t;
    }
    set_class(a);
  }
  // valid output rows of the unit (<= seg) and its first pixel column
  __device__ __forceinline__ int rows(int seg) const {
    const int n = n_class - q * seg;
    return n < 0 ? 0 : (n > seg ? seg : n);
  }
  __device__ __forceinline__ int j0() const { return s * kTileM; }
};

// The MMAs of one input row: for each horizontal tap kx and K step ks one M=128 MMA, fully
// unrolled for a compile-time count of K steps.  The issuing warp then runs no per-MMA loop
// arithmetic between the MMAs (measured: such arithmetic slows the issue of small-N MMAs by
// about a third).  A offsets: kx*a_kx + ks*a_ks (16-byte units); B blocks BBLK16 apart.
template <int PREC, int NKS, int BBLK16, int MAXK>
__device__ __forceinline__ void issue_row(uint32_t d_col, uint64_t a_st, uint64_t b_row, uint32_t idesc,
                                          const uint32_t (&a_off)[3][MAXK], uint32_t leader) {
  static_assert(NKS <= MAXK, "K steps beyond the precomputed offsets");
#pragma unroll
  for (int kx = 0; kx < 3; ++kx)
#pragma unroll
    for (int ks = 0; ks < NKS; ++ks)
      umma_if<PREC>(d_col, a_st + a_off[kx][ks], b_row + (uint64_t)((kx * NKS + ks) * BBLK16), idesc, leader);
}

// Fused 1x1 heads of the last layer for one pixel (Sec. 3.2): h_k = b_k + sum_c w_kc v_c with
// p = sigmoid(h_0) (the logit is also stored when requested), h_1..h_4 as they are, and the
// uncertainty heads h_5..h_8 (NH = 9) through softplus.  Maps are [T][NH][H][W].
template <int CO, int NH>
__device__ __forceinline__ void heads_out(const TcKArgs& a, const float (&v)[CO], int t, size_t px, size_t plane) {
#pragma unroll
  for (int h = 0; h < NH; ++h) {
    float acc = a.head_b[h];
#pragma unroll
    for (int c = 0; c < CO; ++c) acc = fmaf(a.head_w[h * CO + c], v[c], acc);
    if (h == 0) {
      if (a.logits) a.logits[(size_t)t * plane + px] = acc;
      acc = 1.0f / (1.0f + expf(-acc));
    } else if (h >= kHeads) {
      acc = softplus_f(acc);
    }
    a.maps[((size_t)t * NH + h) * plane + px] = acc;
  }
}

template <int CI, int CO, int PREC, bool LAST, bool DGRAD = false, bool PAIR = false>
__global__ void __launch_bounds__(kThreads, PAIR ? 2 : 1) k_dconv_tc(const __grid_constant__ CUtensorMap tmap,
                                                                      const TcKArgs a) {
  using Cfg = TcCfg<CI, CO, PREC, PAIR>;
  // K-dependent sizes: compile-time constants, or the arguments' values for CI = 0
  const int nks = CI > 0 ? Cfg::NKS : a.nks;
  const int g_in = CI > 0 ? Cfg::G : a.g_in;
  const int g_planes = CI > 0 ? Cfg::GP : a.g_planes;
  const uint32_t bimg_bytes = CI > 0 ? (uint32_t)Cfg::BIMG : a.bimg_bytes;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // carve shared memory (1024-aligned base)
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* s_bimg = smem;
  uint8_t* s_stage = smem + ((bimg_bytes + 1023u) & ~1023u);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(s_stage + (size_t)a.nstages * a.stage_bytes);
  // barriers: full[nst], empty[nst], acc_full[SEG], acc_empty[SEG], drain
  constexpr int SEG = Cfg::SEG;
  uint64_t* full_bar = s_bar;
  uint64_t* empty_bar = s_bar + a.nstages;
  uint64_t* accf_bar = empty_bar + a.nstages;
  uint64_t* acce_bar = accf_bar + SEG;
  uint64_t* drain_bar = acce_bar + SEG;
  volatile uint32_t* s_tmem = reinterpret_cast<volatile uint32_t*>(drain_bar + 1);
  volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // input rows per waiter -> MMA handoff: 4, or 2 when the ring is shallower than 8 stages
  // (the protocol needs a ring of at least two handoff groups)
  const int hand_rows = a.nstages >= 8 ? 4 : 2;
  // this CTA's contiguous range of units
  const uint32_t u_begin = (uint32_t)(((unsigned long long)blockIdx.x * a.units) / gridDim.x);
  const uint32_t u_end = (uint32_t)(((unsigned long long)(blockIdx.x + 1) * a.units) / gridDim.x);

  // ---- set-up: weights -> shared, zero pad planes, barriers, TMEM
  {
    const uint4* src = reinterpret_cast<const uint4*>(a.bimg);
    uint4* dst = reinterpret_cast<uint4*>(s_bimg);
    for (int k = threadIdx.x; k < (int)(bimg_bytes / 16); k += kThreads) dst[k] = src[k];
    if (g_planes > g_in) {  // planes beyond the stored groups stay zero (K padding)
      for (int s = 0; s < a.nstages; ++s) {
        uint4* z = reinterpret_cast<uint4*>(s_stage + (size_t)s * a.stage_bytes + (size_t)g_in * a.plane_stride);
        int n16 = (g_planes - g_in) * a.plane_stride / 16;
        for (int k = threadIdx.x; k < n16; k += kThreads) z[k] = make_uint4(0, 0, 0, 0);
      }
    }
    if (threadIdx.x == 0) {
      for (int s = 0; s < a.nstages; ++s) {
        mbar_init(smem_u32(&full_bar[s]), 1);
        mbar_init(smem_u32(&empty_bar[s]), 1);
      }
      for (int s = 0; s < SEG; ++s) {
        mbar_init(smem_u32(&accf_bar[s]), 1);
        mbar_init(smem_u32(&acce_bar[s]), kEpiWarps * 32);
      }
      mbar_init(smem_u32(&drain_bar[0]), 1);
      *s_abort = 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32((const void*)s_tmem)),
                   "r"(Cfg::TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
  }
  const uint32_t tmem = *s_tmem;
  // accumulator start values: every row position holds the bias (in accumulator units)
  float acc0[CO];
#pragma unroll
  for (int c = 0; c < CO; ++c)
    acc0[c] = PREC == kFP8 ? a.bias[c] / a.deq[c] : (DGRAD ? 0.0f : (a.bias_dev ? a.bias_dev[c] : a.bias[c]));
  if (warp < kEpiWarps) {
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    for (int k = 0; k < SEG; ++k)
#pragma unroll
      for (int c = 0; c < CO; c += 16) tmem_st16(lane_addr + Cfg::BASE0 - (uint32_t)(CO * k) + c, acc0 + c);
    tmem_st_wait();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();

  if (warp == 4) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
      const uint32_t nst = (uint32_t)a.nstages;
      uint32_t st = 0, ph = 0, issued = 0;  // stage, phase of its current use, loads issued
      bool ok = (int)blockIdx.x != a.poison_cta;  // a poisoned CTA loads nothing (failure-path test)
      UnitCursor uc;
      uc.init(a, u_begin);
      for (uint32_t u = u_begin; u < u_end && ok; ++u, uc.next(a)) {
        const int n_out = uc.rows(SEG), t = uc.t, j0 = uc.j0(), phi = uc.phi, q = uc.q;
        for (int kk = 0; kk < n_out + 2 && n_out > 0; ++kk) {
          // the slot was released by the MMA that read its previous load (skip on first use)
          if (issued >= nst && !mbar_wait(smem_u32(&empty_bar[st]), ph ^ 1u, a.err, s_abort, a.wait_ns)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&full_bar[st]);
          mbar_expect_tx(fb, a.tx_bytes);
          const int row = phi + (q * SEG + kk - 1) * a.d;
          const int x0 = PREC == kFP8 && a.pair_off >= 0 ? (j0 - a.d - a.pair_off) / 2 : j0 - a.d;
          tma_load_5d(smem_u32(s_stage + (size_t)st * a.stage_bytes), &tmap, 0, x0, 0, row, t, fb);
          ++issued;
          if (++st == nst) {
            st = 0;
            ph ^= 1u;
          }
        }
      }
      // drain: make sure no load of ours is still landing in shared memory
      const uint32_t n_drain = issued < nst ? issued : nst;
      for (uint32_t k = 0; k < n_drain; ++k) {
        // walk back over the last n_drain loads: stage st-1-k with its phase
        const uint32_t back = k + 1;
        const uint32_t s2 = (st + nst - (back % nst)) % nst;
        const uint32_t p2 = (back > st) ? (ph ^ 1u) : ph;
        mbar_wait_own(smem_u32(&full_bar[s2]), p2, a.err, s_abort);
      }
    }
  } else if (warp == 5) {
    // ------------------------------------------------------------ MMA issuer
    // The whole warp runs the loop and lane 0 issues (predicated, no divergence).  It never
    // waits on an mbarrier itself: a shared-memory read whose result this thread consumes
    // waits behind its in-flight MMAs and empties the MMA queue (measured: about 300 cycles
    // per input row).  The waiter warp does the waits and hands over through a named barrier
    // once per hand_rows rows.
    const uint32_t leader = lane == 0 ? 1u : 0u;
    {
      // Descriptors are computed once: the start-address field (bits 0-13, 16-byte units)
      // is advanced by plain addition, which cannot carry out of the field because every
      // shared-memory address is below 256 KB.
      // BF16: 32-byte swizzled rows, one plane per K step; FP8: 16-byte rows, two planes per step
      const uint64_t a_desc0 =
          PREC == kBF16 ? smem_desc(smem_u32(s_stage), 16u, 256u, 6u)
                        : smem_desc(smem_u32(s_stage) + 16u * (uint32_t)(a.pair_off > 0 ? a.pair_off : 0),
                                    a.plane_stride, 128u);
      const uint64_t b_desc0 = smem_desc(smem_u32(s_bimg), 128u, 256u);
      // A offsets in 16-byte units: tap kx starts kx*d pixel rows later, K step ks one plane
      // (BF16) or two planes (FP8) further
      const uint32_t a_kx = PREC == kBF16 ? (uint32_t)(2 * a.d) : (uint32_t)a.d;
      const uint32_t a_ks = PREC == kBF16 ? (a.plane_stride >> 4) : (a.plane_stride >> 3);
      const uint32_t stage16 = a.stage_bytes >> 4;
      const uint32_t nst = (uint32_t)a.nstages;
      // The whole row loop is instantiated per count of K steps and selected once per CTA:
      // a per-row branch on it cost about 200 cycles per row (its jump-table load waits
      // behind the MMAs in flight, like any load this thread consumes).
      auto mma_loop = [&](auto nk_c) {
        constexpr int NK = decltype(nk_c)::value;
        // every (kx, ks) offset once per CTA, kept in registers (the row loop only adds them)
        uint32_t a_off[3][NK];
#pragma unroll
        for (int kx = 0; kx < 3; ++kx)
#pragma unroll
          for (int ks = 0; ks < NK; ++ks) a_off[kx][ks] = (uint32_t)kx * a_kx + (uint32_t)ks * a_ks;
        uint32_t st = 0;             // stage of the current row
        uint64_t a_st = a_desc0;     // descriptor of the current stage
        uint32_t hand = 0;           // handoffs taken
        bool issued = false;
        UnitCursor uc;
        uc.init(a, u_begin);
        for (uint32_t u = u_begin; u < u_end; ++u, uc.next(a)) {
          const int n_out = uc.rows(SEG);
          if (n_out == 0) continue;
          for (int kk = 0; kk < n_out + 2; ++kk) {
            if ((kk & (hand_rows - 1)) == 0) {
              // the waiter has seen this group's TMA data and TMEM releases complete
              named_sync(1u + (hand & 1u));
              ++hand;
              fence_after_sync();
            }
            // blocks b (output rows kk-b) of this input row that belong to the unit
            const int b_lo = kk - n_out + 1 > 0 ? kk - n_out + 1 : 0;
            const int b_hi = kk < 2 ? kk : 2;
            const int nb = b_hi - b_lo + 1;
            const uint32_t d_col = tmem + Cfg::BASE0 - (uint32_t)(CO * kk) + (uint32_t)(CO * b_lo);
            const uint32_t b_sub = (uint32_t)(2 * CO * b_lo);  // 32*CO*b_lo bytes in 16-byte units
            const uint32_t idesc_n = nb == 3 ? Cfg::IDESC3 : (nb == 2 ? Cfg::IDESC2 : Cfg::IDESC1);
            issue_row<PREC, NK, (Cfg::BBLK >> 4)>(d_col, a_st, b_desc0 + b_sub, idesc_n, a_off, leader);
            issued = true;
            if (kk >= 2 && kk - 2 < n_out) umma_commit_if(smem_u32(&accf_bar[kk - 2]), leader);
            umma_commit_if(smem_u32(&empty_bar[st]), leader);
            if (++st == nst) {
              st = 0;
              a_st = a_desc0;
            } else {
              a_st += stage16;
            }
          }
        }
        if (issued && leader) {  // all MMAs of this CTA complete before TMEM is released
          umma_commit(smem_u32(&drain_bar[0]));
          mbar_wait_own(smem_u32(&drain_bar[0]), 0, a.err, s_abort);
        }
      };
      if constexpr (CI > 0) {
        mma_loop(std::integral_constant<int, Cfg::NKS>{});
      } else {
        switch (nks) {
          case 1: mma_loop(std::integral_constant<int, 1>{}); break;
          case 2: mma_loop(std::integral_constant<int, 2>{}); break;
          case 3: mma_loop(std::integral_constant<int, 3>{}); break;
          case 4: mma_loop(std::integral_constant<int, 4>{}); break;
          case 5: mma_loop(std::integral_constant<int, 5>{}); break;
          case 6: mma_loop(std::integral_constant<int, 6>{}); break;
          case 7: mma_loop(std::integral_constant<int, 7>{}); break;
          default: mma_loop(std::integral_constant<int, 8>{}); break;
        }
      }
      __syncwarp();
    }
  } else if (warp == 6) {
    // ------------------------------------------------------------ waiter
    // For each group of hand_rows input rows (groups never span units): wait until their TMA
    // data has landed and, for rows that open an output row position used before, until the
    // epilogue has released those TMEM columns; then arrive on the group's named barrier.
    // It arrives exactly once per group whatever happens (after an abort its waits return at
    // once), so the MMA warp never blocks for good.  Before arriving for group h it waits for
    // the MMA's empty-stage commit of group h-2's first row: the MMA warp has then passed
    // group h-2's sync, so each named barrier has at most one pending arrival.
    const uint32_t nst = (uint32_t)a.nstages;
    uint32_t st = 0, ph = 0;             // stage and fill phase of the current row
    uint32_t used = 0, par = 0;          // row positions used before / parity of their last release
    uint32_t hand = 0;
    uint32_t g_st0 = 0, g_ph0 = 0, g_st1 = 0, g_ph1 = 0;  // first row of the last two groups (even, odd)
    UnitCursor uc;
    uc.init(a, u_begin);
    for (uint32_t u = u_begin; u < u_end; ++u, uc.next(a)) {
      const int n_out = uc.rows(SEG);
      if (n_out == 0) continue;
      for (int k0 = 0; k0 < n_out + 2; k0 += hand_rows) {
        if (lane == 0) {
          const bool odd = hand & 1u;
          if (hand >= 2)
            mbar_wait_own(smem_u32(&empty_bar[odd ? g_st1 : g_st0]), odd ? g_ph1 : g_ph0, a.err, s_abort);
          if (odd) {
            g_st1 = st;
            g_ph1 = ph;
          } else {
            g_st0 = st;
            g_ph0 = ph;
          }
          const int k1 = k0 + hand_rows < n_out + 2 ? k0 + hand_rows : n_out + 2;
          for (int kk = k0; kk < k1; ++kk) {
            mbar_wait(smem_u32(&full_bar[st]), ph, a.err, s_abort, a.wait_ns);
            if (kk < n_out && ((used >> kk) & 1u)) mbar_wait(smem_u32(&acce_bar[kk]), (par >> kk) & 1u, a.err, s_abort, a.wait_ns);
            if (++st == nst) {
              st = 0;
              ph ^= 1u;
            }
          }
        }
        __syncwarp();
        named_arrive(1u + (hand & 1u));
        ++hand;
      }
      // positions 0..n_out-1 were used once more: flip the parity of those used before
      const uint32_t m = (1u << n_out) - 1u;
      par ^= m & used;
      used |= m;
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 0-3)
    const int m = warp * 32 + lane;  // TMEM lane = pixel within the strip
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t fpar = 0;  // per row position: phase of its acc_full barrier for the next use
    bool ok = true;
    // output buffer: groups per pixel row and the first group this layer writes
    const int out_gt = CI > 0 ? Cfg::GO : a.out_gt;
    const int out_g0 = CI > 0 ? 0 : a.out_g0;
    const size_t plane = (size_t)a.H * a.W;
    UnitCursor uc;
    uc.init(a, u_begin);
    for (uint32_t u = u_begin; u < u_end && ok; ++u, uc.next(a)) {
      const int n_out = uc.rows(SEG), t = uc.t, j0 = uc.j0(), phi = uc.phi, q = uc.q;
#pragma unroll 1
      for (int k = 0; k < n_out; ++k) {
        // DGRAD: the ReLU mask of this output row is issued before the accumulator wait, so its
        // DRAM latency overlaps the row's MMAs instead of stalling the conversion below
        uint4 mk[DGRAD ? Cfg::GO : 1][2];
        if (PREC == kBF16 && DGRAD) {
          const int i = phi + (q * SEG + k) * a.d;
          const int j = j0 + m;
          if (j < a.W) {
#pragma unroll
            for (int gq = 0; gq < Cfg::GO; ++gq) {
              const uint4* mp = reinterpret_cast<const uint4*>(
                  a.mask + ((((size_t)t * a.H + i) * out_gt + out_g0 + gq) * a.W + j) * 32);
              mk[gq][0] = __ldcs(mp);
              mk[gq][1] = __ldcs(mp + 1);
            }
          }
        }
        if (!mbar_wait(smem_u32(&accf_bar[k]), (fpar >> k) & 1u, a.err, s_abort, a.wait_ns)) {
          ok = false;
          break;
        }
        fence_after_sync();
        float v[CO];
        const uint32_t col = Cfg::BASE0 - (uint32_t)(CO * k);
#pragma unroll
        for (int c = 0; c < CO; c += 16) tmem_ld16(lane_addr + col + c, v + c);
        tmem_ld_wait();
#pragma unroll
        for (int c = 0; c < CO; c += 16) tmem_st16(lane_addr + col + c, acc0 + c);  // next use starts at the bias
        tmem_st_wait();
        fence_before_sync();
        mbar_arrive(smem_u32(&acce_bar[k]));
        const int i = phi + (q * SEG + k) * a.d;
        const int j = j0 + m;
        if (j >= a.W) continue;
        // the accumulator already holds the bias; FP8 dequantises, the BF16 path fuses the ReLU
        // into its conversion
        if (PREC == kFP8) {
#pragma unroll
          for (int c = 0; c < CO; ++c) v[c] *= a.deq[c];
        }
        if (LAST || PREC == kFP8) {
#pragma unroll
          for (int c = 0; c < CO; ++c) v[c] = fmaxf(v[c], 0.0f);
        }
        if (LAST) {
          const size_t px = (size_t)i * a.W + j;
          // the head count is uniform across the grid: one fully unrolled loop per count
          if (a.nh == kHeads)
            heads_out<CO, kHeads>(a, v, t, px, plane);
          else
            heads_out<CO, kMaxHeads>(a, v, t, px, plane);
        } else if (PREC == kBF16 && DGRAD) {
          // input gradient of the layer below: dz = v * [a > 0] with a that layer's (ReLU) output
#pragma unroll
          for (int gq = 0; gq < Cfg::GO; ++gq) {
            const size_t off = ((((size_t)t * a.H + i) * out_gt + out_g0 + gq) * a.W + j) * 32;
            const uint32_t* mw = reinterpret_cast<const uint32_t*>(mk[gq]);
            uint4 o[2];
            uint32_t* ow = reinterpret_cast<uint32_t*>(o);
#pragma unroll
            for (int e = 0; e < 8; ++e) ow[e] = bf16x2_masked(v[16 * gq + 2 * e], v[16 * gq + 2 * e + 1], mw[e]);
            uint4* dst = reinterpret_cast<uint4*>(a.out + off);
            __stcs(dst, o[0]);
            __stcs(dst + 1, o[1]);
          }
        } else if (PREC == kBF16) {
#pragma unroll
          for (int gq = 0; gq < Cfg::GO; ++gq) {
            uint4 o[2];
            uint32_t* ow = reinterpret_cast<uint32_t*>(o);
#pragma unroll
            for (int e = 0; e < 8; ++e) ow[e] = bf16x2_relu(v[16 * gq + 2 * e], v[16 * gq + 2 * e + 1]);
            uint4* dst = reinterpret_cast<uint4*>(a.out + ((((size_t)t * a.H + i) * out_gt + out_g0 + gq) * a.W + j) * 32);
            __stcs(dst, o[0]);  // streaming: the next layer reads it from HBM anyway; keep L2 for halos
            __stcs(dst + 1, o[1]);
          }
        } else {
#pragma unroll
          for (int gq = 0; gq < Cfg::GO; ++gq) {
            uint4 o;
            uint16_t* oh = reinterpret_cast<uint16_t*>(&o);
#pragma unroll
            for (int e = 0; e < 8; ++e)
              oh[e] = __nv_cvt_float2_to_fp8x2(
                  make_float2(v[16 * gq + 2 * e] * a.out_inv_scale, v[16 * gq + 2 * e + 1] * a.out_inv_scale),
                  __NV_SATFINITE, __NV_E4M3);
            __stcs(reinterpret_cast<uint4*>(a.out + ((((size_t)t * a.H + i) * out_gt + out_g0 + gq) * a.W + j) * 16), o);
          }
        }
      }
      fpar ^= (1u << n_out) - 1u;
    }
  }

  fence_before_sync();
  __syncthreads();
  if (warp == 5) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::TMEM_COLS) : "memory");
  }
}

// ------------------------------------------------------------------ UMMA self-test
// One 128 x N x K product: A [128][K] and B [N][K] pre-packed by the host in the same
// layouts the conv and layer 1 use (A: planes of [128 rows][16 bytes]; B: the per-block
// image).  PREC kBF16, kFP8 or kTF32.
template <int PREC>
__global__ void __launch_bounds__(128, 1) k_umma_selftest(const uint8_t* A, const uint8_t* B, float* D, int N, int K,
                                                          int d_col, int* err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int ES = PREC == kBF16 ? 2 : (PREC == kTF32 ? 4 : 1);
  constexpr int KSTEP = 32 / ES;  // elements per MMA: two 16-byte core-matrix columns
  const int a_bytes = 128 * K * ES, b_bytes = N * K * ES;
  uint8_t* sA = smem;
  uint8_t* sB = smem + a_bytes;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sB + b_bytes);
  volatile uint32_t* s_tmem = reinterpret_cast<volatile uint32_t*>(bar + 1);
  volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);
  for (int k = threadIdx.x; k < a_bytes / 16; k += 128) reinterpret_cast<uint4*>(sA)[k] = reinterpret_cast<const uint4*>(A)[k];
  for (int k = threadIdx.x; k < b_bytes / 16; k += 128) reinterpret_cast<uint4*>(sB)[k] = reinterpret_cast<const uint4*>(B)[k];
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(bar), 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32((const void*)s_tmem)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *s_tmem + (uint32_t)d_col;
  const uint32_t plane = 128 * 16;  // A plane stride: 128 rows x 16 bytes
  const uint32_t bblk = (N / 8) * 256;
  if (threadIdx.x == 0) {
    const uint32_t idesc = instr_desc(PREC, 128, N);
    for (int ks = 0; ks < K / KSTEP; ++ks) {
      uint64_t ad = smem_desc(smem_u32(sA) + 2 * ks * plane, plane, 128);
      uint64_t bd = smem_desc(smem_u32(sB) + ks * bblk, 128, 256);
      umma<PREC>(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
    }
    umma_commit(smem_u32(bar));
  }
  __syncwarp();
  bool ok = mbar_wait(smem_u32(bar), 0, err, s_abort);
  fence_after_sync();
  const int warp = threadIdx.x >> 5;
  if (ok) {
    for (int c = 0; c < N; c += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c, v);
      tmem_ld_wait();
      for (int k = 0; k < 16; ++k) D[(size_t)threadIdx.x * N + c + k] = v[k];
    }
  }
  fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem - (uint32_t)d_col), "r"(512) : "memory");
  }
}

// One M x N x K product with both operands MN-major (the layout of the weight-gradient
// contraction, whose K is pixels): A and B arrive as host-built images of 32-byte-swizzled
// planes, plane g = [K rows][16 elements of M (or N) 16g..16g+15] (the row-planar stage
// layout read along its pixels), planes a_plane / b_plane bytes apart; B's descriptor starts
// b_shift rows into its planes (the tap shift of the contraction).  D: all 128 TMEM lanes x N
// columns read back as float32 [128][N] (for M = 64, the lanes the MMA did not write read
// back whatever TMEM held; the caller finds the data layout).
__global__ void __launch_bounds__(128, 1) k_umma_mn_selftest(const uint8_t* A, const uint8_t* B, float* D, int M,
                                                             int N, int K, int a_bytes, int b_bytes, int a_plane,
                                                             int b_plane, int b_shift, int* err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + ((a_bytes + 1023) & ~1023);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sB + ((b_bytes + 1023) & ~1023));
  volatile uint32_t* s_tmem = reinterpret_cast<volatile uint32_t*>(bar + 1);
  volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);
  for (int k = threadIdx.x; k < a_bytes / 16; k += 128) reinterpret_cast<uint4*>(sA)[k] = reinterpret_cast<const uint4*>(A)[k];
  for (int k = threadIdx.x; k < b_bytes / 16; k += 128) reinterpret_cast<uint4*>(sB)[k] = reinterpret_cast<const uint4*>(B)[k];
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(bar), 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32((const void*)s_tmem)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *s_tmem;
  {  // zero the accumulator columns of every lane, so lanes the MMA does not write read 0
    float z[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) z[k] = 0.0f;
    const int warp = threadIdx.x >> 5;
    for (int c = 0; c < N; c += 16) tmem_st16(tmem + ((uint32_t)(warp * 32) << 16) + c, z);
    tmem_st_wait();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (threadIdx.x == 0) {
    // kind::f16, bf16 inputs, F32 accumulate, A and B MN-major (bits 15, 16)
    const uint32_t idesc = instr_desc(kBF16, M, N) | (1u << 15) | (1u << 16);
    for (int ks = 0; ks < K / 16; ++ks) {
      const uint64_t ad = smem_desc(smem_u32(sA) + ks * 512, (uint32_t)a_plane, 256u, 6u);
      const uint64_t bd = smem_desc(smem_u32(sB) + (b_shift + ks * 16) * 32, (uint32_t)b_plane, 256u, 6u);
      umma<kBF16>(tmem, ad, bd, idesc, 1u);
    }
    umma_commit(smem_u32(bar));
  }
  __syncwarp();
  bool ok = mbar_wait(smem_u32(bar), 0, err, s_abort);
  fence_after_sync();
  const int warp = threadIdx.x >> 5;
  if (ok) {
    for (int c = 0; c < N; c += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c, v);
      tmem_ld_wait();
      for (int k = 0; k < 16; ++k) D[(size_t)threadIdx.x * N + c + k] = v[k];
    }
  }
  fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

size_t tc_smem_bytes(uint32_t bimg_bytes, int seg, int nstages, uint32_t stage_bytes) {
  size_t b = 1024;                                 // alignment slack
  b += (bimg_bytes + 1023u) & ~1023u;              // weights
  b += (size_t)nstages * stage_bytes;              // stages
  b += 8 * (2 * nstages + 2 * seg + 1) + 16;       // barriers, tmem addr, abort flag
  return b;
}

constexpr size_t kSmemBudget = 227 * 1024;
constexpr size_t kPairSmemBudget = 112 * 1024;  // per CTA when two CTAs share an SM
std::mutex g_tc_launch_mutex;  // serialises attribute-set + launch of the conv kernels

// Row sizes of a layer with ci input channels at dilation d.
struct TcSizes {
  int nks, g_in, g_planes;
  uint32_t bimg_bytes, plane_stride, tx_bytes, stage_bytes;
};
TcSizes tc_sizes(int ci, int co, int d, int prec) {
  TcSizes z;
  const int kstep = prec == kBF16 ? 16 : 32;
  z.nks = (ci + kstep - 1) / kstep;
  z.g_in = ci / 16;
  z.g_planes = prec == kBF16 ? z.g_in : 2 * z.nks;
  z.bimg_bytes = (uint32_t)(3 * z.nks * 3 * (co / 8) * 256);
  z.plane_stride = (uint32_t)tc_box_width(d) * (prec == kBF16 ? 32u : 16u);  // box width: a multiple of 32
  z.tx_bytes = (uint32_t)z.g_in * z.plane_stride;
  z.stage_bytes = ((uint32_t)z.g_planes * z.plane_stride + 1023u) & ~1023u;
  return z;
}

int tc_seg(int co) { return (512 / co - 2) < kMaxSeg ? (512 / co - 2) : kMaxSeg; }

template <int CI, int CO, int PREC, bool LAST, bool DGRAD = false, bool PAIR = false>
cudaError_t launch_tc_impl(const TcLayerArgs& la, int num_sms, cudaStream_t s) {
  using Cfg = TcCfg<CI, CO, PREC, PAIR>;
  constexpr size_t budget = PAIR ? kPairSmemBudget : kSmemBudget;
  const int ci = CI > 0 ? CI : la.ci;
  if (la.co != CO || ci != la.ci || ci < 16 || ci > kTcMaxCin || ci % 16) return cudaErrorInvalidValue;
  TcKArgs a{};
  a.bimg = static_cast<const uint8_t*>(la.bimg);
  for (int c = 0; c < CO; ++c) {
    a.bias[c] = la.bias ? la.bias[c] : 0.0f;
    a.deq[c] = la.deq ? la.deq[c] : 1.0f;
  }
  if (LAST) {
    if (la.nh != kHeads && la.nh != kMaxHeads) return cudaErrorInvalidValue;
    a.nh = la.nh;
    for (int k = 0; k < la.nh; ++k) {
      a.head_b[k] = la.head_b[k];
      for (int c = 0; c < CO; ++c) a.head_w[k * CO + c] = la.head_w[k * CO + c];
    }
  }
  a.out_inv_scale = la.out_inv_scale;
  a.out = static_cast<uint8_t*>(la.out);
  a.maps = la.maps;
  a.logits = la.logits;
  a.T = la.T;
  a.H = la.H;
  a.W = la.W;
  a.d = la.d;
  a.NS = (la.W + kTileM - 1) / kTileM;
  int rows0 = (la.H + la.d - 1) / la.d;
  a.NQ = (rows0 + Cfg::SEG - 1) / Cfg::SEG;
  const long long units = (long long)la.T * a.NS * la.d * a.NQ;
  if (units >= (1LL << 31)) return cudaErrorInvalidValue;
  a.units = (uint32_t)units;
  const TcSizes z = tc_sizes(ci, CO, la.d, PREC);
  a.nks = z.nks;
  a.g_in = z.g_in;
  a.g_planes = z.g_planes;
  a.bimg_bytes = z.bimg_bytes;
  a.plane_stride = z.plane_stride;
  a.tx_bytes = z.tx_bytes;
  a.stage_bytes = z.stage_bytes;
  a.out_g0 = la.out_g0;
  a.out_gt = la.out_gt;
  a.bias_dev = la.bias_dev;
  a.mask = static_cast<const uint8_t*>(la.mask);
  a.wait_ns = la.wait_ns ? la.wait_ns : kWaitLimitNs;
  a.poison_cta = la.poison_cta;
  a.pair_off = (PREC == kFP8 && la.pair_rows) ? (la.d & 1) : -1;
  if (DGRAD && (!a.mask || PREC != kBF16 || LAST)) return cudaErrorInvalidValue;
  if (CI > 0 && !LAST && (la.out_g0 != 0 || la.out_gt != Cfg::GO)) return cudaErrorInvalidValue;
  if (!LAST && (la.out_g0 < 0 || la.out_g0 + Cfg::GO > la.out_gt)) return cudaErrorInvalidValue;
  a.err = la.err;
  if (a.units == 0) return cudaSuccess;
  int nst = la.stages > 0 ? la.stages : kMaxStages;
  if (nst < kMinStages) return cudaErrorInvalidValue;
  while (nst > kMinStages && tc_smem_bytes(z.bimg_bytes, Cfg::SEG, nst, z.stage_bytes) > budget) --nst;
  a.nstages = nst;
  size_t smem = tc_smem_bytes(z.bimg_bytes, Cfg::SEG, nst, z.stage_bytes);
  if (smem > budget) return cudaErrorInvalidConfiguration;
  // the limit is this launch's size, which differs between the layers that share the
  // runtime-K instance: set and launch under one lock, so that contexts on several host
  // threads never launch under another launch's smaller limit
  std::lock_guard<std::mutex> lock(g_tc_launch_mutex);
  cudaError_t e = cudaFuncSetAttribute(k_dconv_tc<CI, CO, PREC, LAST, DGRAD, PAIR>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long ctas = (PAIR ? 2LL : 1LL) * num_sms;  // persistent: every CTA resident at once
  const long long grid = (long long)a.units < ctas ? (long long)a.units : ctas;
  k_dconv_tc<CI, CO, PREC, LAST, DGRAD, PAIR><<<(unsigned)grid, kThreads, smem, s>>>(*la.tmap, a);
  return cudaGetLastError();
}

}  // namespace

int tc_box_width(int d) { return (kTileM + 2 * d + 31) / 32 * 32; }

size_t tc_bimg_bytes(int ci, int co, int prec) { return tc_sizes(ci, co, 1, prec).bimg_bytes; }

bool tc_layer_fits(int ci, int co, int d, int prec) {
  if (ci < 16 || ci > kTcMaxCin || ci % 16 || co < 16 || co > 64 || co % 16) return false;
  const TcSizes z = tc_sizes(ci, co, d, prec);
  return tc_smem_bytes(z.bimg_bytes, tc_seg(co), kMinStages, z.stage_bytes) <= kSmemBudget;
}

// B image: for horizontal tap kx and k-step ks, one [N = 3 CO][K = kstep] block whose rows are
// n = ky*CO + co (the three vertical taps side by side), in no-swizzle K-major core-matrix
// order: byte (n/8)*256 + (k/EPG)*128 + (n%8)*16 + (k%EPG)*esize.  Input channels beyond CI
// (FP8 padding) are zero.  FP8 weights are divided by w_scale[co].
void tc_pack_bimg(const float* w /*[9][CI][CO] tap, ci, co*/, int CI, int CO, int prec, const float* w_scale,
                  void* dst) {
  const int kstep = prec == kBF16 ? 16 : 32;
  const int epg = prec == kBF16 ? 8 : 16;
  const int es = prec == kBF16 ? 2 : 1;
  const int nks = (CI + kstep - 1) / kstep;
  const size_t bblk = (size_t)3 * (CO / 8) * 256;
  uint8_t* out = static_cast<uint8_t*>(dst);
  for (int kx = 0; kx < 3; ++kx)
    for (int ks = 0; ks < nks; ++ks) {
      uint8_t* blk = out + ((size_t)kx * nks + ks) * bblk;
      for (int n = 0; n < 3 * CO; ++n) {
        const int ky = n / CO, co = n % CO, tap = ky * 3 + kx;
        for (int k = 0; k < kstep; ++k) {
          int ci = ks * kstep + k;
          float v = ci < CI ? w[((size_t)tap * CI + ci) * CO + co] : 0.0f;
          size_t off = (size_t)(n / 8) * 256 + (size_t)(k / epg) * 128 + (size_t)(n % 8) * 16 + (size_t)(k % epg) * es;
          if (prec == kBF16) {
            __nv_bfloat16 h = __float2bfloat16_rn(v);
            memcpy(blk + off, &h, 2);
          } else {
            float sv = v / w_scale[co];
            blk[off] = (uint8_t)__nv_cvt_float_to_fp8(sv, __NV_SATFINITE, __NV_E4M3);
          }
        }
      }
    }
}

// Plain layers (ci == co, output filling whole pixel rows of its buffer) and every last layer
// run the compile-time instances; layers of dense blocks and of the U-Net (ci != co, or an
// output that is a channel range of a wider buffer) run the runtime-K instances.
// Two CTAs per SM (PAIR instances) for the 32- and 48-channel FP8 layers, every 32- or
// 48-channel last layer and the runtime-K layers with 16 or 32 output channels (dense blocks,
// U-Net; measured: FP8 dense-block net 27.9k -> 37.1k frames/s), when a ring of kMinStages
// stages fits half of the shared memory.  Measured on the 256-frame
// batch of the 48-channel net: FP8 middle layers 0.429 -> 0.365 ms, last layer 0.590 -> 0.515
// ms (FP8) and 0.606 -> 0.529 ms (BF16).  The BF16 middle layers keep one CTA per SM: at half
// the shared memory their ring shrinks to 4 stages and the launch went 0.618 -> 0.702 ms.
static bool tc_use_pair(const TcLayerArgs& a, bool last) {
  const bool plain = a.ci == a.co && a.out_g0 == 0 && a.out_gt == a.co / 16;
  if (!last && !plain) {  // runtime-K layers (dense blocks, U-Net): 16 or 32 output channels
    if (a.co != 16 && a.co != 32) return false;
  } else if ((a.prec != kFP8 && !last) || (a.co != 32 && a.co != 48) || a.ci != a.co) {
    return false;
  }
  const TcSizes z = tc_sizes(a.ci, a.co, a.d, a.prec);
  const int seg = kPairTmemCols / a.co < kMaxSeg ? kPairTmemCols / a.co : kMaxSeg;
  return tc_smem_bytes(z.bimg_bytes, seg, kMinStages, z.stage_bytes) <= kPairSmemBudget;
}

cudaError_t launch_dconv_tc(const TcLayerArgs& a, bool last, int num_sms, cudaStream_t s) {
  const bool plain = a.ci == a.co && a.out_g0 == 0 && a.out_gt == a.co / 16;
  if (last || plain) {
    if (a.ci != a.co) return cudaErrorInvalidValue;
    if (tc_use_pair(a, last)) {
      const bool bf = a.prec == kBF16;
      if (a.co == 32)
        return bf ? launch_tc_impl<32, 32, kBF16, true, false, true>(a, num_sms, s)
                  : (last ? launch_tc_impl<32, 32, kFP8, true, false, true>(a, num_sms, s)
                          : launch_tc_impl<32, 32, kFP8, false, false, true>(a, num_sms, s));
      return bf ? launch_tc_impl<48, 48, kBF16, true, false, true>(a, num_sms, s)
                : (last ? launch_tc_impl<48, 48, kFP8, true, false, true>(a, num_sms, s)
                        : launch_tc_impl<48, 48, kFP8, false, false, true>(a, num_sms, s));
    }
#define SML_TC(CC)                                                                                          \
  case CC:                                                                                                  \
    if (a.prec == kBF16)                                                                                    \
      return last ? launch_tc_impl<CC, CC, kBF16, true>(a, num_sms, s) : launch_tc_impl<CC, CC, kBF16, false>(a, num_sms, s); \
    else                                                                                                    \
      return last ? launch_tc_impl<CC, CC, kFP8, true>(a, num_sms, s) : launch_tc_impl<CC, CC, kFP8, false>(a, num_sms, s);
    switch (a.co) {
      SML_TC(16)
      SML_TC(32)
      SML_TC(48)
      SML_TC(64)
    }
#undef SML_TC
    return cudaErrorInvalidValue;
  }
  const bool bf = a.prec == kBF16;
  if (tc_use_pair(a, false)) {
    if (a.co == 16)
      return bf ? launch_tc_impl<0, 16, kBF16, false, false, true>(a, num_sms, s)
                : launch_tc_impl<0, 16, kFP8, false, false, true>(a, num_sms, s);
    return bf ? launch_tc_impl<0, 32, kBF16, false, false, true>(a, num_sms, s)
              : launch_tc_impl<0, 32, kFP8, false, false, true>(a, num_sms, s);
  }
  switch (a.co) {
    case 16: return bf ? launch_tc_impl<0, 16, kBF16, false>(a, num_sms, s) : launch_tc_impl<0, 16, kFP8, false>(a, num_sms, s);
    case 32: return bf ? launch_tc_impl<0, 32, kBF16, false>(a, num_sms, s) : launch_tc_impl<0, 32, kFP8, false>(a, num_sms, s);
    case 48: return bf ? launch_tc_impl<0, 48, kBF16, false>(a, num_sms, s) : launch_tc_impl<0, 48, kFP8, false>(a, num_sms, s);
    case 64: return bf ? launch_tc_impl<0, 64, kBF16, false>(a, num_sms, s) : launch_tc_impl<0, 64, kFP8, false>(a, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_dconv_tc_train(const TcLayerArgs& a, bool dgrad, int num_sms, cudaStream_t s) {
  if (a.prec != kBF16 || a.ci != a.co || a.out_g0 != 0 || a.out_gt != a.co / 16) return cudaErrorInvalidValue;
  switch (a.co) {
    case 16: return dgrad ? launch_tc_impl<16, 16, kBF16, false, true>(a, num_sms, s) : launch_tc_impl<16, 16, kBF16, false>(a, num_sms, s);
    case 32: return dgrad ? launch_tc_impl<32, 32, kBF16, false, true>(a, num_sms, s) : launch_tc_impl<32, 32, kBF16, false>(a, num_sms, s);
    case 48: return dgrad ? launch_tc_impl<48, 48, kBF16, false, true>(a, num_sms, s) : launch_tc_impl<48, 48, kBF16, false>(a, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_umma_mn_selftest(const void* A, const void* B, float* D, int M, int N, int K, int a_bytes,
                                    int b_bytes, int a_plane, int b_plane, int b_shift, int* err, cudaStream_t s) {
  if ((M != 64 && M != 128) || N < 16 || N > 256 || N % 16 || K < 16 || K % 16 || a_bytes % 1024 || b_bytes % 1024 ||
      a_plane % 256 || b_plane % 256 || b_shift < 0)
    return cudaErrorInvalidValue;
  // the operands' descriptors stay inside the images: A reads M/16 planes of K rows, B M/16
  // planes of b_shift + K rows
  if ((long long)(M / 16 - 1) * a_plane + (long long)K * 32 > a_bytes ||
      (long long)(N / 16 - 1) * b_plane + (long long)(b_shift + K) * 32 > b_bytes)
    return cudaErrorInvalidValue;
  const size_t smem = 1024 + (size_t)a_bytes + (size_t)b_bytes + 64;
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_umma_mn_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_umma_mn_selftest<<<1, 128, smem, s>>>(static_cast<const uint8_t*>(A), static_cast<const uint8_t*>(B), D, M, N, K,
                                          a_bytes, b_bytes, a_plane, b_plane, b_shift, err);
  return cudaGetLastError();
}

cudaError_t launch_umma_selftest(const void* A, const void* B, float* D, int N, int K, int prec, int d_col, int* err,
                                 cudaStream_t s) {
  const int es = prec == kBF16 ? 2 : (prec == kTF32 ? 4 : 1);
  size_t smem = 1024 + (size_t)128 * K * es + (size_t)N * K * es + 64;
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  if (prec == kBF16) {
    cudaError_t e = cudaFuncSetAttribute(k_umma_selftest<kBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_umma_selftest<kBF16><<<1, 128, smem, s>>>(static_cast<const uint8_t*>(A), static_cast<const uint8_t*>(B), D, N, K, d_col, err);
  } else if (prec == kTF32) {
    cudaError_t e = cudaFuncSetAttribute(k_umma_selftest<kTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_umma_selftest<kTF32><<<1, 128, smem, s>>>(static_cast<const uint8_t*>(A), static_cast<const uint8_t*>(B), D, N, K, d_col, err);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_umma_selftest<kFP8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_umma_selftest<kFP8><<<1, 128, smem, s>>>(static_cast<const uint8_t*>(A), static_cast<const uint8_t*>(B), D, N, K, d_col, err);
  }
  return cudaGetLastError();
}

}  // namespace sml
