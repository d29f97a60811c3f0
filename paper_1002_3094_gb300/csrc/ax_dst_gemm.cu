// Sine transform along z as a dense GEMM on the tcgen05 tensor cores, for the
// FP32 working precision of the mixed method (the z-transform of the
// preconditioner of Section 4.2, Eq. fft_phi, written as a matrix product):
//
//     out[l] = sum_k in[k] S[k][l],   S[k][l] = sqrt(2/L) sin(pi (k+1) (l+1) / L),
//     L = nz + 1 (0-based k, l < nz).
//
// Even / odd split.  S[k][n-1-l] = (-1)^k S[k][l], so with
//     P[l] = sum_{k even} in[k] S[k][l],   Q[l] = sum_{k odd} in[k] S[k][l]
// for l < ceil(n/2):  out[l] = P[l] + Q[l],  out[n-1-l] = P[l] - Q[l]
// (once for the middle column of odd n).  Two GEMMs of half the width and half
// the depth replace one full one: half the multiply-adds.  The input arrives
// with its even columns stored first (the split layout of ax_common.cuh).
//
// Precision.  The input arrives split, in = hi + lo, hi = bf16(in),
// lo = bf16(in - hi) (|in - hi - lo| <= 2^-17 |in|), and S as S_hi = bf16(S),
// S_lo = bf16(S - S_hi).  The products hi S_hi + lo S_hi (and, with `three`,
// + hi S_lo) accumulate in FP32 in the tensor memory.  Without the third
// product the transform multiplies by S_hi: a fixed symmetric matrix within
// ~3e-3 (spectral norm) of S, so the preconditioner S_hi T^-1 S_hi is still
// symmetric positive definite and close to B^-1; with it the transform is S
// to about 2^-16.  Either way the FP64 residual replacement keeps the
// solution accuracy.
//
// Tiles: 128 rows x 128 columns l of both P and Q per CTA (256 TMEM columns;
// persistent CTAs keep two tiles in flight, 512 columns, so that the epilogue
// of one overlaps the MMAs of the next), K in blocks of 64 (the even blocks
// feed P, the odd ones Q) through a ring of shared-memory stages (4 of 48 KB,
// or 3 of 64 KB with S_lo), each filled by bulk copies (cp.async.bulk) of one
// 32 KB input tile (hi and lo halves) and one or two 16 KB tiles of S (stored
// in the same layout: row l, column k).  Warp roles: warp
// 0 lane 0 issues tcgen05.mma (M = 128, N = 128, K = 16, BF16 x BF16 -> FP32);
// warp 1 lane 0 issues the copies; warps 4..7 run the epilogue (tcgen05.ld,
// the even / odd combination, global stores, optional (r, out) partial).
// Every mbarrier wait is bounded; on expiry the CTA records the failure in
// *err, stops issuing work, waits (bounded) for its MMAs and frees its TMEM.
#include <cuda_bf16.h>
#include <cstdint>
#include <cstring>
#include <cmath>
#include <algorithm>
#include <vector>
#include "ax_common.cuh"

namespace ax {

namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64;
// one tile: P and Q, kBN columns each; two tiles in flight (MMA / epilogue)
constexpr unsigned kTileCols = 2 * kBN;
constexpr unsigned kTmemCols = 2 * kTileCols;
constexpr int kATileBytes = kSplitTileBytes;                // hi and lo halves, 32 KB
constexpr int kBTileBytes = kBN * kBK * 2;                  // 16 KB
constexpr int kEpiWarps = 8;                                // warps 4 .. 11
constexpr int kGemmThreads = 128 + 32 * kEpiWarps;
constexpr unsigned kWaitPolls = 1u << 22;

template <int THREE> struct GemmStages {
  static constexpr int stage_bytes = kATileBytes + (1 + THREE) * kBTileBytes;
  static constexpr int stages = THREE ? 3 : 4;
};

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: canonical K-major layout without swizzle.
// Core matrices of 8 rows x 16 bytes (128 contiguous bytes); the two core
// matrices of one K = 16 step are 128 bytes apart (leading byte offset), and
// consecutive 8-row groups 1024 bytes apart (stride byte offset; a tile row
// group holds the 8 core matrices of K = 64).  Bits 46-47: descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(const void *p) {
  const unsigned a = smem_u32(p);
  return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(1024u >> 4) << 32) |
         (1ull << 46);
}
// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28.
constexpr unsigned kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(kBN >> 3) << 17) |
                            ((unsigned)(kBM >> 4) << 24);

__device__ __forceinline__ void umma(unsigned d_tmem, uint64_t a, uint64_t b, unsigned accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 TMEM lanes x 32 consecutive 32-bit columns: thread i of the warp gets
// lane (base + i), columns col .. col + 31.
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32]) {
  unsigned r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Tiles in shared memory: byte offset of element (row, k) of a K = 64 block is
// (row / 8) 1024 + (k / 8) 128 + (row % 8) 16 + (k % 8) 2.

// Tile t (persistent CTAs take t = blockIdx.x, + gridDim.x, ...): N tile
// fastest, so the CTAs working on one M tile at a time share its input tiles
// in L2.  The tiles run from the last right-hand side to the first: the
// kernels that write this transform's input (the update pass, the mode
// solves) and read its output (the mode solves) go from the first to the
// last, so the input written last, still in L2, is read first, and the output
// written last is read first by the next kernel.
__device__ __forceinline__ void gemm_tile(const GemmDstArgs &a, int t, int &m, int &mt, int &nt) {
  t = a.m * a.mtiles * a.ntiles - 1 - t;
  nt = t % a.ntiles;
  const int mm = t / a.ntiles;
  m = mm / a.mtiles;
  mt = mm - m * a.mtiles;
}

template <int THREE>
__global__ void __launch_bounds__(kGemmThreads, 1) dst_gemm_kernel(const GemmDstArgs a) {
  constexpr int kStageBytes = GemmStages<THREE>::stage_bytes;
  constexpr int kStages = GemmStages<THREE>::stages;
  extern __shared__ __align__(1024) unsigned char gsm_raw[];
  unsigned char *gsm =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], tfull_bar[2], tempty_bar[2];
  __shared__ unsigned tmem_base;
  __shared__ int abort_flag;
  __shared__ double red[kEpiWarps];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int KB = a.ktiles;
  const unsigned polls = a.polls ? a.polls : kWaitPolls;
  const int ntile_all = a.m * a.mtiles * a.ntiles;
  if (a.gate != nullptr && *a.gate == 0) return;  // nothing selected: before any set-up

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull_bar[b], 1);
      mbar_init(&tempty_bar[b], kEpiWarps);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tmem_base;

  if (warp == 0) {
    // ---- MMA issuer ----
    if (lane == 0) {
      bool ok = true;
      int kk = 0;  // k blocks consumed so far (ring position)
      int it = 0;  // tiles processed so far (TMEM buffer = it & 1)
      for (int t = blockIdx.x; t < ntile_all && ok; t += gridDim.x) {
        int m, mt, nt;
        gemm_tile(a, t, m, mt, nt);
        if (!rhs_selected(a.st, a.mask, m)) continue;  // skipped alike by every role
        const int b = it & 1;
        // the epilogue must have drained this buffer (its previous tile)
        if (it >= 2 && !mbar_wait(&tempty_bar[b], (unsigned)((it >> 1) - 1) & 1u, polls)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const unsigned accP = tmem + (unsigned)b * kTileCols, accQ = accP + kBN;
        for (int kb = 0; kb < KB; ++kb, ++kk) {
          const int s = kk % kStages;
          if (!mbar_wait(&full_bar[s], (unsigned)(kk / kStages) & 1u, polls)) {
            ok = false;
            break;
          }
          tc_fence_after();
          unsigned char *st = gsm + s * kStageBytes;
          const bool odd = kb >= a.kbe;  // Q block
          const unsigned acc_t = odd ? accQ : accP;
          const int first = odd ? a.kbe : 0;
#pragma unroll
          for (int j = 0; j < kBK / 16; ++j) {
            const uint64_t ahi = smem_desc(st + j * 256), alo = smem_desc(st + kATileBytes / 2 + j * 256);
            const uint64_t bhi = smem_desc(st + kATileBytes + j * 256);
            umma(acc_t, ahi, bhi, (kb != first || j != 0) ? 1u : 0u);
            umma(acc_t, alo, bhi, 1u);
            if (THREE) umma(acc_t, ahi, smem_desc(st + kATileBytes + kBTileBytes + j * 256), 1u);
          }
          umma_commit(&empty_bar[s]);
        }
        if (ok) umma_commit(&tfull_bar[b]);  // accumulators of this tile complete
        ++it;
      }
      if (!ok) {
        atomicExch(&abort_flag, 1);
        if (a.err) atomicExch(a.err, 1);
      }
    }
  } else if (warp == 1) {
    // ---- bulk copies: input tile (m, mt, kb) and the S tiles (nt, kb) ----
    if (lane == 0) {
      int kk = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntile_all && ok; t += gridDim.x) {
        int m, mt, nt;
        gemm_tile(a, t, m, mt, nt);
        if (!rhs_selected(a.st, a.mask, m)) continue;
        const unsigned char *ga = a.A + ((size_t)m * a.mtiles + mt) * KB * (size_t)kATileBytes;
        const unsigned char *gb =
            reinterpret_cast<const unsigned char *>(a.SB) + (size_t)nt * KB * 2 * kBTileBytes;
        for (int kb = 0; kb < KB; ++kb, ++kk) {
          const int s = kk % kStages;
          if (kk >= kStages && !mbar_wait(&empty_bar[s], (unsigned)(kk / kStages - 1) & 1u, polls)) {
            ok = false;
            break;
          }
          if (abort_flag || kk == a.stall_at) {  // stall_at: test of the expiry path, see GemmDstArgs
            ok = false;
            break;
          }
          unsigned char *st = gsm + s * kStageBytes;
          mbar_arrive_tx(&full_bar[s], (unsigned)(kATileBytes + (1 + THREE) * kBTileBytes));
          bulk_g2s(st, ga + (size_t)kb * kATileBytes, kATileBytes, &full_bar[s]);
          bulk_g2s(st + kATileBytes, gb + (size_t)kb * 2 * kBTileBytes, kBTileBytes, &full_bar[s]);
          if (THREE)
            bulk_g2s(st + kATileBytes + kBTileBytes, gb + ((size_t)kb * 2 + 1) * kBTileBytes, kBTileBytes,
                     &full_bar[s]);
        }
      }
      if (!ok) {
        atomicExch(&abort_flag, 1);
        if (a.err) atomicExch(a.err, 1);
        // wait (bounded) for the copies this warp issued before it stopped:
        // only the last kStages issues can still be in flight
        for (int j = kk > kStages ? kk - kStages : 0; j < kk; ++j)
          mbar_wait(&full_bar[j % kStages], (unsigned)(j / kStages) & 1u, polls);
      }
    }
  } else if (warp >= 4) {
    // ---- epilogue: TMEM -> registers -> global (and the (r, out) partial) ----
    // warp w drains TMEM lane quarter w % 4, columns half (w - 4) / 4 of P and Q
    const int ew = warp - 4;
    const int q = warp & 3, half = ew >> 2;
    // per epilogue warp a 32 x 32 FP32 transpose tile behind the stages
    float *epi = reinterpret_cast<float *>(gsm + kStages * kStageBytes);
    const int n = a.n, ne = (n + 1) >> 1;
    int it = 0;  // tiles processed so far, as counted by the MMA issuer
    for (int t = blockIdx.x; t < ntile_all; t += gridDim.x) {
      int m, mt, nt;
      gemm_tile(a, t, m, mt, nt);
      if (!rhs_selected(a.st, a.mask, m)) continue;
      const int b = it & 1;
      ++it;
      const bool ok = !abort_flag && mbar_wait(&tfull_bar[b], (unsigned)((it - 1) >> 1) & 1u, polls);
      if (!ok) {
        atomicExch(&abort_flag, 1);
        if (a.err) atomicExch(a.err, 1);
      }
      tc_fence_after();
      const int grow = mt * kBM + q * 32 + lane;
      // row scale of this lane's row (1 without rowscale)
      const float rsc = (a.rowscale != nullptr && grow < a.nr) ? __ldg(a.rowscale + m * a.rsstride + grow) : 1.f;
      float acc = 0.f;
      if (__all_sync(0xffffffffu, ok)) {
        const size_t roff = (size_t)m * (size_t)a.field + (size_t)grow * a.pitch;
        const bool pupd = a.pa != nullptr;
        float *outr = pupd ? nullptr : a.out + roff;
        const float *rr = (a.r != nullptr) ? a.r + roff : nullptr;
        // direction update: p_new = out + beta p_old (and x += alpha p_old)
        float *por = nullptr, *pnr = nullptr, *xr = nullptr;
        const float *pog = nullptr;
        float *png = nullptr, *xg = nullptr;
        float beta = 0.f, alpha = 0.f;
        if (pupd) {
          const bool odd = a.st[m].iters & 1;
          pog = odd ? a.pb : a.pa;
          png = odd ? a.pa : a.pb;
          por = const_cast<float *>(pog) + roff;
          pnr = png + roff;
          beta = (float)a.st[m].beta;
          if (a.x != nullptr) {
            xg = a.x;
            xr = a.x + roff;
            alpha = (float)a.st[m].alpha;
          }
        }
        const unsigned tP = tmem + ((unsigned)(q * 32) << 16) + (unsigned)b * kTileCols;
#pragma unroll 1
        for (int c = half * 2; c < half * 2 + 2; ++c) {
          const int l0 = nt * kBN + c * 32;
          if (!__any_sync(0xffffffffu, grow < a.nr) || l0 >= ne) break;  // nothing left for this warp
          if (a.tout) {
            // mode-major output: lane = row, so every store of the warp is a run
            // of 32 consecutive rows of one column (no transpose needed)
            float P[32], Q[32];
            tmem_ld32(tP + (unsigned)(c * 32), P);
            if (a.ktiles > a.kbe) {
              tmem_ld32(tP + (unsigned)(kBN + c * 32), Q);
            } else {
#pragma unroll
              for (int i = 0; i < 32; ++i) Q[i] = 0.f;  // n = 1: no odd column
            }
            if (grow < a.nr) {
              float *ob = a.out + (size_t)m * n * a.tpitch + grow;
#pragma unroll
              for (int i = 0; i < 32; ++i) {
                const int l = l0 + i;
                if (l < ne) {
                  if (a.cosfwd) {  // even output columns from P, odd ones from Q
                    ob[(size_t)(2 * l) * a.tpitch] = rsc * P[i];
                    if (2 * l + 1 < n) ob[(size_t)(2 * l + 1) * a.tpitch] = rsc * Q[i];
                  } else {
                    ob[(size_t)l * a.tpitch] = rsc * (P[i] + Q[i]);
                    const int lm = n - 1 - l;
                    if (lm != l) ob[(size_t)lm * a.tpitch] = rsc * (P[i] - Q[i]);
                  }
                }
              }
            }
            continue;
          }
          if (rr == nullptr) {
            // Write-back transposed through this warp's 32 x 32 shared tile
            // (XOR-swizzled: conflict-free in both directions), so that every
            // global access of the warp is a run of 32 consecutive columns of
            // one row: first the columns l0 + j (P + Q), then their mirrors
            // n - 1 - l0 - j (P - Q; the accumulators are read from TMEM again
            // so that neither pass holds them).  The cosine forward writes
            // P to the even columns 2 (l0 + j) and Q to the odd ones.  The direction update loads
            // 16 rows of p_old and x before it uses them, so that the warp has
            // 32 loads in flight at once.
            float *T = epi + ew * 1024;
            const int row0 = mt * kBM + q * 32;
            const size_t mbase = (size_t)m * (size_t)a.field;
#pragma unroll 1
            for (int pass = 0; pass < 2; ++pass) {
              {
                float P[32], Q[32];
                tmem_ld32(tP + (unsigned)(c * 32), P);
                if (a.ktiles > a.kbe) {
                  tmem_ld32(tP + (unsigned)(kBN + c * 32), Q);
                } else {
#pragma unroll
                  for (int i = 0; i < 32; ++i) Q[i] = 0.f;  // n = 1: no odd column
                }
                if (a.cosfwd) {  // even output columns from P, odd ones from Q
#pragma unroll
                  for (int i = 0; i < 32; ++i) T[lane * 32 + (i ^ lane)] = rsc * (pass ? Q[i] : P[i]);
                } else {
#pragma unroll
                  for (int i = 0; i < 32; ++i) T[lane * 32 + (i ^ lane)] = rsc * (pass ? P[i] - Q[i] : P[i] + Q[i]);
                }
              }
              __syncwarp();
              const int lc = l0 + lane;  // column of the half range
              // output column: the mirrored pair l, n - 1 - l (the middle column of
              // odd n once), or for the cosine forward 2 l and 2 l + 1
              const int col = a.cosfwd ? 2 * lc + pass : (pass ? n - 1 - lc : lc);
              const bool colok = a.cosfwd ? (lc < ne && col < n) : (lc < ne && (pass == 0 || col != lc));
              const size_t cbase = mbase + (size_t)row0 * a.pitch + col;
              if (pupd) {
#pragma unroll 1
                for (int h = 0; h < 32; h += 16) {
                  float po[16], xv[16];
#pragma unroll
                  for (int j = 0; j < 16; ++j) {
                    const int r = h + j;
                    const bool ok = colok && row0 + r < a.nr;
                    po[j] = ok ? __ldg(pog + cbase + (size_t)r * a.pitch) : 0.f;
                    xv[j] = (ok && xg) ? xg[cbase + (size_t)r * a.pitch] : 0.f;
                  }
#pragma unroll
                  for (int j = 0; j < 16; ++j) {
                    const int r = h + j;
                    if (colok && row0 + r < a.nr) {
                      const size_t e = cbase + (size_t)r * a.pitch;
                      png[e] = fmaf(beta, po[j], T[r * 32 + (lane ^ r)]);
                      if (xg) xg[e] = fmaf(alpha, po[j], xv[j]);
                    }
                  }
                }
              } else {
#pragma unroll 8
                for (int r = 0; r < 32; ++r)
                  if (colok && row0 + r < a.nr) a.out[cbase + (size_t)r * a.pitch] = T[r * 32 + (lane ^ r)];
              }
              __syncwarp();
            }
            continue;
          }
          float P[32], Q[32];
          tmem_ld32(tP + (unsigned)(c * 32), P);
          if (a.ktiles > a.kbe) {
            tmem_ld32(tP + (unsigned)(kBN + c * 32), Q);
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) Q[i] = 0.f;  // n = 1: no odd column
          }
          if (grow < a.nr) {
#pragma unroll
            for (int i = 0; i < 32; i += 4) {
              const int l = l0 + i;
              float s0[4], d0[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                s0[e] = rsc * (P[i + e] + Q[i + e]);  // out[l + e]
                d0[e] = rsc * (P[i + e] - Q[i + e]);  // out[n - 1 - l - e]
              }
              if (l + 3 < ne && (n & 3) == 0) {
                // n % 4 == 0: both runs are whole aligned float4 groups, and the
                // mirrored one (columns n - 4 - l .. n - 1 - l) lies above ne
                const int lm = n - 4 - l;
                if (pupd) {
                  const float4 pa4 = *reinterpret_cast<const float4 *>(por + l);
                  const float4 pb4 = *reinterpret_cast<const float4 *>(por + lm);
                  *reinterpret_cast<float4 *>(pnr + l) =
                      make_float4(fmaf(beta, pa4.x, s0[0]), fmaf(beta, pa4.y, s0[1]), fmaf(beta, pa4.z, s0[2]),
                                  fmaf(beta, pa4.w, s0[3]));
                  *reinterpret_cast<float4 *>(pnr + lm) =
                      make_float4(fmaf(beta, pb4.x, d0[3]), fmaf(beta, pb4.y, d0[2]), fmaf(beta, pb4.z, d0[1]),
                                  fmaf(beta, pb4.w, d0[0]));
                  if (xr) {
                    float4 xa = *reinterpret_cast<const float4 *>(xr + l);
                    float4 xb = *reinterpret_cast<const float4 *>(xr + lm);
                    xa.x = fmaf(alpha, pa4.x, xa.x); xa.y = fmaf(alpha, pa4.y, xa.y);
                    xa.z = fmaf(alpha, pa4.z, xa.z); xa.w = fmaf(alpha, pa4.w, xa.w);
                    xb.x = fmaf(alpha, pb4.x, xb.x); xb.y = fmaf(alpha, pb4.y, xb.y);
                    xb.z = fmaf(alpha, pb4.z, xb.z); xb.w = fmaf(alpha, pb4.w, xb.w);
                    *reinterpret_cast<float4 *>(xr + l) = xa;
                    *reinterpret_cast<float4 *>(xr + lm) = xb;
                  }
                } else {
                  *reinterpret_cast<float4 *>(outr + l) = make_float4(s0[0], s0[1], s0[2], s0[3]);
                  *reinterpret_cast<float4 *>(outr + lm) = make_float4(d0[3], d0[2], d0[1], d0[0]);
                }
                if (rr) {
                  const float4 ra = *reinterpret_cast<const float4 *>(rr + l);
                  const float4 rb = *reinterpret_cast<const float4 *>(rr + lm);
                  acc = fmaf(ra.x, s0[0], acc); acc = fmaf(ra.y, s0[1], acc);
                  acc = fmaf(ra.z, s0[2], acc); acc = fmaf(ra.w, s0[3], acc);
                  acc = fmaf(rb.x, d0[3], acc); acc = fmaf(rb.y, d0[2], acc);
                  acc = fmaf(rb.z, d0[1], acc); acc = fmaf(rb.w, d0[0], acc);
                }
              } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  const int le = l + e, lm = n - 1 - le;
                  if (le < ne) {
                    if (pupd) {
                      const float po = por[le];
                      pnr[le] = fmaf(beta, po, s0[e]);
                      if (xr) xr[le] = fmaf(alpha, po, xr[le]);
                    } else {
                      outr[le] = s0[e];
                    }
                    if (rr) acc = fmaf(rr[le], s0[e], acc);
                    if (lm != le) {  // the middle column of odd n is written once
                      if (pupd) {
                        const float po = por[lm];
                        pnr[lm] = fmaf(beta, po, d0[e]);
                        if (xr) xr[lm] = fmaf(alpha, po, xr[lm]);
                      } else {
                        outr[lm] = d0[e];
                      }
                      if (rr) acc = fmaf(rr[lm], d0[e], acc);
                    }
                  }
                }
              }
            }
          }
        }
      }
      // buffer b drained: the MMA issuer may reuse it
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty_bar[b]);
      if (a.partial) {
        const double sw = warp_sum((double)acc);
        if (lane == 0) red[ew] = sw;
        asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");
        if (ew == 0 && lane == 0) {
          double tot = 0.0;
#pragma unroll
          for (int i = 0; i < kEpiWarps; ++i) tot += red[i];
          a.partial[(size_t)m * kPartialStride + mt * a.ntiles + nt] = tot;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    // every MMA this CTA issued has completed once its tile's tfull fired; after
    // an expired wait, give the tensor core a bounded moment before freeing
    if (abort_flag) {
      for (int b = 0; b < 2; ++b) mbar_wait(&tfull_bar[b], 0u, polls);
    }
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace

size_t dst_gemm_smem_bytes(int three) {
  constexpr size_t kEpiBytes = (size_t)kEpiWarps * 32 * 32 * sizeof(float);  // transpose tiles
  return (three ? (size_t)GemmStages<1>::stages * GemmStages<1>::stage_bytes
                : (size_t)GemmStages<0>::stages * GemmStages<0>::stage_bytes) +
         kEpiBytes + 1024;
}

// K tiles of even and of odd input columns.  The writers of the split operand
// store whole 8-column chunks, so the ranges cover n rounded up to 8 columns
// (positions past n hold zeros; S has zero rows there).
int dst_gemm_kbe(int n) { return (((n + 7) & ~7) / 2 + kBK - 1) / kBK; }
int dst_gemm_ktiles(int n) { return 2 * dst_gemm_kbe(n); }
int dst_gemm_ntiles(int n) { return ((n + 1) / 2 + kBN - 1) / kBN; }
int dst_gemm_mtiles(int rows) { return (rows + kBM - 1) / kBM; }

// S tiles: for every N tile (128 output columns l < ceil(n/2)) and K block (64
// input columns: the even columns 0, 2, ... in the first kbe blocks, the odd
// ones after) a 16 KB tile of S_hi and one of S_lo, each in the shared-memory
// layout above holding S[k][l] at (row l, column k).  Values in FP64, rounded
// to BF16 (nearest, ties to even, by way of FP32).
std::vector<uint16_t> dst_gemm_table(int n, int kind) {
  const int KB = dst_gemm_ktiles(n), KBE = dst_gemm_kbe(n), NT = dst_gemm_ntiles(n);
  const int L = n + 1, ne = (n + 1) / 2;
  auto to_bf16 = [](double x) -> uint16_t {
    const float v = (float)x;
    uint32_t u;
    std::memcpy(&u, &v, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
  };
  auto from_bf16 = [](uint16_t h) -> double {
    const uint32_t u = (uint32_t)h << 16;
    float v;
    std::memcpy(&v, &u, 4);
    return v;
  };
  // orthonormal cosine matrix C[l][k] = c_l sqrt(2/n) cos(pi (2k + 1) l / (2n)),
  // c_0 = 1/sqrt 2, the integer (2k + 1) l reduced exactly mod 4n
  auto cosm = [n](int l, int k) -> double {
    const long long e = ((long long)(2 * k + 1) * l) % (4LL * n);
    return std::sqrt(2.0 / n) * (l == 0 ? std::sqrt(0.5) : 1.0) * std::cos(M_PI * (double)e / (2.0 * n));
  };
  const size_t tile = (size_t)kBN * kBK;  // elements of one 32 KB tile
  std::vector<uint16_t> t((size_t)NT * KB * 2 * tile, 0);
  for (int nt = 0; nt < NT; ++nt)
    for (int kb = 0; kb < KB; ++kb) {
      uint16_t *hi = t.data() + ((size_t)nt * KB + kb) * 2 * tile;
      uint16_t *lo = hi + tile;
      const bool second = kb >= KBE;
      for (int nl = 0; nl < kBN; ++nl) {
        const int l = nt * kBN + nl;  // output column of the half range
        if (l >= ne) continue;
        for (int kl = 0; kl < kBK; ++kl) {
          const int kk = (second ? kb - KBE : kb) * kBK + kl;  // position in the K half
          double v;
          if (kind == kTableCosForward) {
            // first half: u_kk = r_kk + r_{n-1-kk} times C[2l][kk]; second half:
            // w_kk = r_kk - r_{n-1-kk} times C[2l+1][kk] (kk < ceil(n/2))
            const int lo_ = second ? 2 * l + 1 : 2 * l;
            if (kk >= ne || lo_ >= n) continue;
            v = cosm(lo_, kk);
          } else {
            const int k = second ? 2 * kk + 1 : 2 * kk;  // input index, even ones first
            if (k >= n) continue;
            if (kind == kTableCosInverse) {
              v = cosm(k, l);  // out[l] = sum over modes k of C[k][l] in[k]
            } else {
              const long long e = ((long long)(k + 1) * (l + 1)) % (2LL * L);  // sin(pi e / L), e reduced
              v = std::sqrt(2.0 / L) * std::sin(M_PI * (double)e / L);
            }
          }
          const uint16_t h = to_bf16(v);
          const int off = ((nl >> 3) * 1024 + (kl >> 3) * 128 + (nl & 7) * 16 + (kl & 7) * 2) / 2;
          hi[off] = h;
          lo[off] = to_bf16(v - from_bf16(h));
        }
      }
    }
  return t;
}

void launch_dst_gemm(const GemmDstArgs &a, cudaStream_t s) {
  const size_t smem = dst_gemm_smem_bytes(a.three);
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  const int tiles = a.m * a.mtiles * a.ntiles;
  dim3 grid(std::min(tiles, sms));
  note_launch();
  if (a.three) {
    ensure_smem_attr((const void *)dst_gemm_kernel<1>, smem);
    dst_gemm_kernel<1><<<grid, kGemmThreads, smem, s>>>(a);
  } else {
    ensure_smem_attr((const void *)dst_gemm_kernel<0>, smem);
    dst_gemm_kernel<0><<<grid, kGemmThreads, smem, s>>>(a);
  }
}

}  // namespace ax
