// Weighted Gram on the 5th-generation tensor cores (Eq. spod-discrete-snapshots):
// M_f = kappa * Qhat_f^* W Qhat_f from BF16 operands (BF16 precision) or from
// the split x = hi + lo (BF16X3 precision), FP32 accumulation in tensor memory.
//
// Real embedding: with Y_f = [Re Qhat_f ; Im Qhat_f] (2nb rows x points, K-major
// in HBM; sqrt(W) is already folded into Qhat), D = Y_f Y_f^T gives
//   Re M_f[l][l'] = D[l][l'] + D[nb+l][nb+l'],  Im M_f[l][l'] = D[l][nb+l'] - D[nb+l][l'].
// An item is two 64-point blocks of one frequency; its stage holds the TMA
// boxes (NP rows x 64 points x 2 blocks, NP = 2nb rounded up to 16, 128-byte
// swizzle) of hi and, for BF16X3, of lo.  Per K step of 16 (N = NP):
//   A1 (+)= hi hi^T   restarted every `flush` blocks (short FP32 runs in the
//                      tensor core), drained into Kahan-compensated registers.
//                      The tensor core's FP32 accumulation rounds toward zero,
//                      so a run of R MMAs carries a relative bias of about
//                      R * 2^-24 on the positive diagonal; measured on the
//                      512 x 256 x 3 jet grid, the mean diagonal bias was
//                      -2e-7 / -6e-7 / -3e-6 / -1.4e-5 for runs of 2 / 4 / 16 / 64
//                      blocks.  Runs are therefore short (one or two blocks);
//   A2 (+)= hi lo^T   BF16X3, one run per frequency segment (2^-8 of D, so its
//                      tensor-core rounding is far below the FP32 level of D),
//                      read once when the segment ends;
// and Y Y^T = A1 + A2 + A2^T + lo lo^T, with lo hi^T = (hi lo^T)^T taken in FP64
// when the partials are collected.  Of lo lo^T (2^-16 of D) only the diagonal
// sum_p lo_r[p]^2 is kept, summed by two warps straight from the staged lo
// tiles: its off-diagonal entries are sums of uncorrelated rounding products
// (relative size 2^-16 / sqrt(points)), while the diagonal is a bias (about
// 2.4e-6 of D) that would shift small eigenvalues.  A operand rows >= 2nb only
// feed accumulator rows that are never read.
//
// Persistent CTAs (one per SM by default) walk a contiguous range of the
// f-major list of (frequency, block pair) items.  Warp 8 issues TMA into a
// ring of stages, warp 9 issues the MMAs, warps 0-7 drain TMEM (two warps per
// lane quadrant, half of the columns each; quadrants without a row < 2nb
// skip the reads) and warps 10-11 sum the lo squares.  When the CTA's run of
// a frequency ends the sums go to slot (cta + f) (the pairs (cta, f) of
// contiguous ranges are monotone in both, so cta + f is unique);
// k_gram_tc_collect adds the slots of every frequency in CTA order (no
// atomics: bit-reproducible) and k_gram_tc_finish forms M_f.
#include <algorithm>

#include "tc_common.cuh"

namespace spod {
namespace {

constexpr int kMaxStages = 8;
constexpr int kKpb = 2;                   // 64-point blocks per item (one TMA copy per operand)
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kTmaWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1, kDiagWarp0 = kEpiWarps + 2;
constexpr int kDiagThreads = 64;
constexpr int kThreadsGram = (kEpiWarps + 4) * 32;
constexpr uint32_t kTmemCols = 512;       // A1 buffers at columns b * np (b < nacc), then two A2 buffers
constexpr int kMaxAcc = 4;                // A1 accumulator buffers at most

struct GramTcArgs {
  int nb, r2, np, nf;
  int64_t nkb;                            // items (block pairs) per frequency in this chunk
  int64_t nblk;                           // 64-point blocks per frequency in this chunk
  int64_t nitems;                         // nf * nkb
  int flush;                              // 64-point blocks per A1 run
  int nacc;                               // A1 buffers in tensor memory (2..kMaxAcc, as np allows)
  int stall0;                             // self-test: the first item's copies are never issued, so
                                          // every wait on them runs out (the bounded-wait path)
  int nst;                                // pipeline stages
  uint32_t box_bytes;                     // one 64-point block of one operand: NP rows x 128 bytes
};

// Kahan compensated addition: (s, c) += y
__device__ __forceinline__ void kahan_add(float& s, float& c, float y) {
  const float yy = y - c;
  const float t = s + yy;
  c = (t - s) - yy;
  s = t;
}

// The same on two independent pairs with packed FP32x2 instructions (each
// lane rounds to nearest exactly as the scalar form: identical results, half
// the instructions in the drains).
__device__ __forceinline__ void kahan_add2(float& s0, float& s1, float& c0, float& c1, float y0, float y1) {
  asm("{\n"
      " .reg .b64 rs, rc, ry, ryy, rt, rd;\n"
      " mov.b64 rs, {%0, %1};\n"
      " mov.b64 rc, {%2, %3};\n"
      " mov.b64 ry, {%4, %5};\n"
      " sub.rn.f32x2 ryy, ry, rc;\n"
      " add.rn.f32x2 rt, rs, ryy;\n"
      " sub.rn.f32x2 rd, rt, rs;\n"
      " sub.rn.f32x2 rc, rd, ryy;\n"
      " mov.b64 {%0, %1}, rt;\n"
      " mov.b64 {%2, %3}, rc;\n"
      "}"
      : "+f"(s0), "+f"(s1), "+f"(c0), "+f"(c1)
      : "f"(y0), "f"(y1));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

struct GramHdr {
  uint64_t full[kMaxStages], empty[kMaxStages], accfull[kMaxAcc], accempty[kMaxAcc], a2empty[2], drain;
  uint32_t tmem_base;
  int abort;
};

// Walks the group and segment structure of a CTA's range, one 64-point
// block at a time: a segment is the run of one frequency, a group (one A1
// run in tensor memory) at most `flush` consecutive blocks of a segment; a
// group may end inside an item.  All roles step it identically.
struct GroupWalk {
  int fprev = -1;
  int in_group = 0;
  int g = -1, seg = -1;
  int acc = -1, accph = 0;      // the group's A1 buffer and the parity of its use (g / nacc) & 1
  bool sstart = false;
  __device__ __forceinline__ bool step(int f, int flush, int nacc) {   // true when the block starts a group
    sstart = f != fprev;
    const bool start = sstart || in_group == flush;
    if (sstart) ++seg;
    if (start) {
      ++g;
      in_group = 0;
      if (++acc == nacc) { acc = 0; accph ^= 1; }
    }
    ++in_group;
    fprev = f;
    return start;
  }
};

// Position of a CTA's item in the (frequency, block pair) list and in the
// stage ring, advanced without divisions (the issuing threads are on the
// critical path of every item).
struct Cursor {
  int f, kp;          // frequency, block pair within it
  int s, ph;          // stage, parity of the ring pass (i / nst) & 1
  __device__ __forceinline__ void init(int64_t item0, int nkb) {
    f = (int)(item0 / nkb);
    kp = (int)(item0 - (int64_t)f * nkb);
    s = 0;
    ph = 0;
  }
  __device__ __forceinline__ bool last_of_f(int nkb) const { return kp + 1 == nkb; }
  __device__ __forceinline__ void next(int nkb, int nst) {
    if (++kp == nkb) { kp = 0; ++f; }
    if (++s == nst) { s = 0; ph ^= 1; }
  }
};

// Slot layout (bytes): A1 (sum, carry) pairs [r2][r2] float2, A2 [r2][r2]
// float, then the lo-square diagonal [r2] float.
__host__ __device__ inline size_t gram_slot_bytes(int r2) { return (size_t)r2 * r2 * 12 + (size_t)r2 * 4; }

template <bool X3, int HC>
__global__ void __launch_bounds__(kThreadsGram, 1) k_gram_tc(const __grid_constant__ CUtensorMap map_hi,
                                                   const __grid_constant__ CUtensorMap map_lo, GramTcArgs a,
                                                   uint8_t* __restrict__ slots, unsigned* __restrict__ gflags) {
  using namespace tc;
  constexpr int NOPS = X3 ? 2 : 1;
  extern __shared__ unsigned char smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  GramHdr* hdr = reinterpret_cast<GramHdr*>(sm);
  uint8_t* stages = sm + 1024;
  const uint32_t op_bytes = a.box_bytes * kKpb;          // one operand of an item
  const uint32_t stage_bytes = op_bytes * NOPS;          // [hi blocks][lo blocks]

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t i0 = a.nitems * blockIdx.x / gridDim.x;
  const int64_t i1 = a.nitems * (blockIdx.x + 1) / gridDim.x;
  const int nit = (int)(i1 - i0);
  const int FB = a.flush;
  const int nkb = (int)a.nkb, nblk = (int)a.nblk;

  if (tid == 0) {
    for (int i = 0; i < a.nst; ++i) {
      mbar_init(smem_u32(&hdr->full[i]), 1);
      // released by the MMA commit, and for BF16X3 also by the lo-square warps
      mbar_init(smem_u32(&hdr->empty[i]), X3 ? 1 + kDiagThreads : 1);
    }
    for (int i = 0; i < a.nacc; ++i) {
      mbar_init(smem_u32(&hdr->accfull[i]), 1);
      mbar_init(smem_u32(&hdr->accempty[i]), kEpiThreads);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&hdr->a2empty[i]), kEpiThreads);
    }
    mbar_init(smem_u32(&hdr->drain), 1);
    hdr->abort = 0;
    fence_mbar_init();
  }
  if (warp == kMmaWarp) {
    tmem_alloc(smem_u32(&hdr->tmem_base), kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = hdr->tmem_base;
  volatile int* abort_flag = &hdr->abort;

  if (warp == kTmaWarp && lane == 0 && nit > 0) {
    // ---------------- TMA producer
    prefetch_tmap(&map_hi);
    if (X3) prefetch_tmap(&map_lo);
    int issued = 0;
    const int skipped = a.stall0 ? 1 : 0;       // items at the head never issued (self-test)
    Cursor cu;
    cu.init(i0, nkb);
    for (int i = 0; i < nit; ++i, cu.next(nkb, a.nst)) {
      const int s = cu.s;
      if (i >= a.nst && !mbar_wait(smem_u32(&hdr->empty[s]), cu.ph ^ 1, abort_flag, gflags)) break;
      if (i < skipped) {
        issued = i + 1;
        continue;
      }
      const uint32_t fb = smem_u32(&hdr->full[s]);
      mbar_arrive_expect_tx(fb, stage_bytes);
      uint8_t* st = stages + (size_t)s * stage_bytes;
      tma_load_4d(smem_u32(st), &map_hi, 0, 0, cu.f, cu.kp * kKpb, fb);
      if (X3) tma_load_4d(smem_u32(st + op_bytes), &map_lo, 0, 0, cu.f, cu.kp * kKpb, fb);
      issued = i + 1;
    }
    // copies still in flight must land before the CTA can exit
    for (int i = max(skipped, issued - a.nst); i < issued; ++i)
      mbar_drain(smem_u32(&hdr->full[i % a.nst]), (i / a.nst) & 1, gflags);
  } else if (warp == kMmaWarp && lane == 0 && nit > 0) {
    // ---------------- MMA issuer
    const uint32_t idesc = idesc_bf16(128, a.np, 0, 0);
    GroupWalk gw;
    Cursor cu;
    cu.init(i0, nkb);
    bool ok = true;
    for (int i = 0; i < nit && ok; ++i, cu.next(nkb, a.nst)) {
      const int f = cu.f, kp = cu.kp;
      const int s = cu.s;
      if (!mbar_wait(smem_u32(&hdr->full[s]), cu.ph, abort_flag, gflags)) break;
      tc_fence_after();
      const uint32_t st = smem_u32(stages + (size_t)s * stage_bytes);
      // a block past the chunk's points (odd block count) holds no data of this chunk
      const int nvalid = min(kKpb, nblk - kp * kKpb);
      const bool item_last = i + 1 == nit || cu.last_of_f(nkb);
      for (int j = 0; j < nvalid; ++j) {
        const bool gstart = gw.step(f, FB, a.nacc);
        const bool sstart = gw.sstart;              // only on an item's first block
        const int g = gw.g, acc = gw.acc, sg = gw.seg, a2b = sg & 1;
        const bool gend = (item_last && j + 1 == nvalid) || gw.in_group == FB;
        // the buffer's previous run (use (g / nacc) - 1) must have been drained
        if (gstart && g >= a.nacc &&
            !mbar_wait(smem_u32(&hdr->accempty[acc]), gw.accph ^ 1, abort_flag, gflags)) {
          ok = false;
          break;
        }
        if (X3 && sstart && sg >= 2 &&
            !mbar_wait(smem_u32(&hdr->a2empty[a2b]), ((sg >> 1) - 1) & 1, abort_flag, gflags)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d1 = tmem + (uint32_t)(acc * a.np);
        const uint32_t d2 = tmem + (uint32_t)((a.nacc + a2b) * a.np);
        const uint32_t hi = st + (uint32_t)j * a.box_bytes;
        const uint32_t lo = hi + op_bytes;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint64_t dh = sdesc_sw128(hi + k * 32, 16, 1024);
          mma_bf16(d1, dh, dh, idesc, (gstart && k == 0) ? 0u : 1u);                // A1 (+)= hi hi^T
          if (X3) {
            const uint64_t dl = sdesc_sw128(lo + k * 32, 16, 1024);
            mma_bf16(d2, dh, dl, idesc, (sstart && j == 0 && k == 0) ? 0u : 1u);   // A2 (+)= hi lo^T
          }
        }
        if (gend) mma_commit(smem_u32(&hdr->accfull[acc]));
      }
      if (ok) mma_commit(smem_u32(&hdr->empty[s]));
    }
    mma_commit(smem_u32(&hdr->drain));
    mbar_drain(smem_u32(&hdr->drain), 0, gflags);
  } else if (X3 && warp >= kDiagWarp0 && nit > 0) {
    // ---------------- lo-square diagonal of every lo block.  Eight threads
    // share a row (one 16-byte chunk each, so a warp reads 512 contiguous
    // bytes: no bank conflicts); a row's chunks are permuted by the swizzle,
    // which a sum over the row does not see.  Thread t keeps the partial sums
    // of rows t/8 + 8 j in q[j]; the eight partials of a row are combined by
    // shuffles when the CTA's run of a frequency ends.
    const int t = tid - kDiagWarp0 * 32;
    const int rsub = t >> 3, chunk = t & 7;
    constexpr int kRowsPer = 16;                      // rows rsub + 8 j, j < 16: up to 128 rows
    float q[kRowsPer];
#pragma unroll
    for (int j = 0; j < kRowsPer; ++j) q[j] = 0.f;
    Cursor cu;
    cu.init(i0, nkb);
    for (int i = 0; i < nit; ++i, cu.next(nkb, a.nst)) {
      const int f = cu.f, kp = cu.kp;
      const bool send = i + 1 == nit || cu.last_of_f(nkb);
      const int s = cu.s;
      if (!mbar_wait(smem_u32(&hdr->full[s]), cu.ph, abort_flag, gflags)) break;
      const int nvalid = min(kKpb, nblk - kp * kKpb);
      for (int b = 0; b < nvalid; ++b) {
        const uint8_t* lo = stages + (size_t)s * stage_bytes + op_bytes + (size_t)b * a.box_bytes;
#pragma unroll
        for (int j = 0; j < kRowsPer; ++j) {
          const int r = rsub + 8 * j;
          if (r < a.r2) {
            const uint4 w4 = *reinterpret_cast<const uint4*>(lo + (size_t)r * 128 + chunk * 16);
            const uint32_t ws[4] = {w4.x, w4.y, w4.z, w4.w};
            float acc = 0.f;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float la = __uint_as_float(ws[e] << 16), lb = __uint_as_float(ws[e] & 0xFFFF0000u);
              acc = fmaf(la, la, acc);
              acc = fmaf(lb, lb, acc);
            }
            q[j] += acc;
          }
        }
      }
      mbar_arrive(smem_u32(&hdr->empty[s]));
      if (send) {
        float* dg = reinterpret_cast<float*>(slots + ((size_t)blockIdx.x + (size_t)f) * gram_slot_bytes(a.r2) +
                                             (size_t)a.r2 * a.r2 * 12);
#pragma unroll
        for (int j = 0; j < kRowsPer; ++j) {
          float v = q[j];
          v += __shfl_xor_sync(0xffffffffu, v, 1);
          v += __shfl_xor_sync(0xffffffffu, v, 2);
          v += __shfl_xor_sync(0xffffffffu, v, 4);
          const int r = rsub + 8 * j;
          if (chunk == 0 && r < a.r2) dg[r] = v;
          q[j] = 0.f;
        }
      }
    }
  } else if (warp < kEpiWarps) {
    // ---------------- epilogue: TMEM -> registers -> slots.  Warp (quad,
    // half) drains rows quad*32 .. +31 and the HC columns of its half; of A1
    // (symmetric) only the 8-column chunks that reach the upper triangle
    // (some row of the quad <= some column of the chunk) are read and summed.
    constexpr int CH = HC / 8;
    const int quad = warp & 3, half = warp >> 2;
    const int row = quad * 32 + lane;
    const int col0 = half * HC;
    const bool active = quad * 32 < a.r2;         // this lane quadrant holds rows of D
    int nch = 0;                                  // chunks [CH - nch, CH) of this warp are upper-triangle ones
#pragma unroll
    for (int c = 0; c < CH; ++c) nch += (col0 + 8 * c + 7 >= quad * 32) ? 1 : 0;
    const int c_first = CH - nch;
    float s1[HC], c1[HC];
#pragma unroll
    for (int j = 0; j < HC; ++j) { s1[j] = 0.f; c1[j] = 0.f; }
    GroupWalk gw;
    Cursor cu;
    cu.init(i0, nkb);
    bool ok = true;
    for (int i = 0; i < nit && ok; ++i, cu.next(nkb, a.nst)) {
     const int f = cu.f;
     const int nvalid = min(kKpb, nblk - cu.kp * kKpb);
     const bool item_last = i + 1 == nit || cu.last_of_f(nkb);
     for (int j = 0; j < nvalid; ++j) {
      gw.step(f, FB, a.nacc);
      const bool send = item_last && j + 1 == nvalid;
      const bool gend = send || gw.in_group == FB;
      if (!gend) continue;
      const int acc = gw.acc, a2b = gw.seg & 1;
      // one decision per warp: the tcgen05.ld below must be executed by the whole warp
      const bool got = mbar_wait(smem_u32(&hdr->accfull[acc]), gw.accph, abort_flag, gflags);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      tc_fence_after();
      if (active && nch > 0) {
        // this warp's A1 chunks in one batch of loads and one wait
        const uint32_t t1 = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * a.np) + (uint32_t)col0;
        float v[HC];
#pragma unroll
        for (int c = 0; c < CH; ++c)
          if (c >= c_first) tmem_ld8(t1 + (uint32_t)(c * 8), v + c * 8);
        tmem_wait_ld();
        tc_fence_before();
        mbar_arrive(smem_u32(&hdr->accempty[acc]));
#pragma unroll
        for (int c = 0; c < CH; ++c)
          if (c >= c_first) {
#pragma unroll
            for (int e = 0; e < 8; e += 2)
              kahan_add2(s1[c * 8 + e], s1[c * 8 + e + 1], c1[c * 8 + e], c1[c * 8 + e + 1], v[c * 8 + e],
                         v[c * 8 + e + 1]);
          }
      } else {
        tc_fence_before();
        mbar_arrive(smem_u32(&hdr->accempty[acc]));
      }
      if (!send) continue;
      // the CTA's run of frequency f ends: its sums go to slot (cta + f)
      uint8_t* slot = slots + ((size_t)blockIdx.x + (size_t)f) * gram_slot_bytes(a.r2);
      const bool wr = row < a.r2;
      if (active) {
        float2* d1 = reinterpret_cast<float2*>(slot) + (size_t)row * a.r2 + col0;
#pragma unroll
        for (int jj = 0; jj < HC; ++jj) {
          if (wr && col0 + jj < a.r2) d1[jj] = make_float2(s1[jj], c1[jj]);
          s1[jj] = 0.f;
          c1[jj] = 0.f;
        }
      }
      if (X3) {
        if (active) {
          // the segment's A2 (its MMAs completed with the last group's), not symmetric: all of it
          const uint32_t t2 = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)((a.nacc + a2b) * a.np) +
                              (uint32_t)col0;
          float v[HC];
#pragma unroll
          for (int c = 0; c < CH; ++c) tmem_ld8(t2 + (uint32_t)(c * 8), v + c * 8);
          tmem_wait_ld();
          tc_fence_before();
          mbar_arrive(smem_u32(&hdr->a2empty[a2b]));
          float* d2 = reinterpret_cast<float*>(slot + (size_t)a.r2 * a.r2 * 8) + (size_t)row * a.r2 + col0;
#pragma unroll
          for (int jj = 0; jj < HC; ++jj)
            if (wr && col0 + jj < a.r2) d2[jj] = v[jj];
        } else {
          tc_fence_before();
          mbar_arrive(smem_u32(&hdr->a2empty[a2b]));
        }
      }
     }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// CTA c's item range is [floor(c W / G), floor((c+1) W / G)); the CTA holding item i.
__device__ __forceinline__ int64_t cta_of_item(int64_t i, int64_t W, int64_t G) { return ((i + 1) * G - 1) / W; }

// acc[f] (+)= sum over the CTAs c that covered frequency f of slot (c + f), in
// CTA order, of D = A1 + A2 + A2^T + diag(lo lo^T) (A1 as a compensated (sum, carry)
// pair, read from its upper triangle).
__global__ void k_gram_tc_collect(const uint8_t* __restrict__ slots, int r2, int64_t nkb, int64_t G, int x3,
                                  int first, double* __restrict__ acc) {
  const int f = blockIdx.x;
  const int64_t W = (int64_t)gridDim.x * nkb;
  const int64_t c0 = cta_of_item((int64_t)f * nkb, W, G);
  const int64_t c1 = cta_of_item((int64_t)(f + 1) * nkb - 1, W, G);
  double* dst = acc + (int64_t)f * r2 * r2;
  const size_t sb = gram_slot_bytes(r2);
  for (int e = threadIdx.x; e < r2 * r2; e += blockDim.x) {
    const int i = e / r2, j = e - i * r2;
    double v = 0.0;
    for (int64_t c = c0; c <= c1; ++c) {
      const uint8_t* slot = slots + (size_t)(c + f) * sb;
      // A1 is symmetric and only its upper triangle is summed by the epilogue
      const float2 sc = reinterpret_cast<const float2*>(slot)[i <= j ? e : j * r2 + i];
      v += (double)sc.x + (double)sc.y;
      if (x3) {
        const float* a2 = reinterpret_cast<const float*>(slot + (size_t)r2 * r2 * 8);
        v += (double)a2[e] + (double)a2[j * r2 + i];
        if (i == j) v += (double)reinterpret_cast<const float*>(slot + (size_t)r2 * r2 * 12)[i];
      }
    }
    dst[e] = first ? v : dst[e] + v;
  }
}

// M_f from D = Y Y^T: upper triangle formed, kappa applied, Hermitian completion, NaN check.
//
// Folded mean (what != nullptr, r2 = 2 nb + 1): the stored rows are the
// spectra Z of x - c and row 2 nb is rho = sqrt(W) (mu - c); the spectra of
// x - mu are Z - rho What_f, i.e. row i loses rho u_i with u_i = Re What_f
// (i < nb) or Im What_f (nb <= i < 2 nb), so in FP64
//   Dc[i][j] = D[i][j] - u_i D[j][2nb] - u_j D[i][2nb] + u_i u_j D[2nb][2nb].
__global__ void k_gram_tc_finish(const double* __restrict__ acc, int nb, int r2, const double* __restrict__ what,
                                 double kappa, double* __restrict__ gram, unsigned* __restrict__ flags) {
  const int f = blockIdx.x;
  const double* D = acc + (int64_t)f * r2 * r2;
  const double ur = what ? what[2 * f] : 0.0, ui = what ? what[2 * f + 1] : 0.0;
  const int rr = 2 * nb;
  auto dc = [&](int i, int j) -> double {
    double v = D[i * r2 + j];
    if (what) {
      const double u_i = i < nb ? ur : ui, u_j = j < nb ? ur : ui;
      v += u_i * u_j * D[rr * r2 + rr] - u_i * D[j * r2 + rr] - u_j * D[i * r2 + rr];
    }
    return v;
  };
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e - i * nb;
    const int l = min(i, j), lp = max(i, j);
    double vr = dc(l, lp) + dc(nb + l, nb + lp);
    double vi = dc(l, nb + lp) - dc(nb + l, lp);
    vr *= kappa;
    vi *= kappa;
    if (i > j) vi = -vi;
    if (i == j) {
      vi = 0.0;
      if (!isfinite(vr)) atomicOr(flags, FLAG_NAN);
    }
    double* o = gram + (((int64_t)f * nb + i) * nb + j) * 2;
    o[0] = vr;
    o[1] = vi;
  }
}

size_t gram_tc_smem_stages(const spod_plan_s& p, int nst) {
  const int nops = p.desc.precision == SPOD_PREC_BF16X3 ? 2 : 1;
  const size_t np = (size_t)((2 * p.nb + 15) / 16 * 16);
  // + the rows an M = 128 A operand reads past the last stage's last block
  return 1024 + 1024 + (size_t)nst * nops * kKpb * np * 128 + (128 - np) * 128;
}

template <bool X3, int HC>
cudaError_t launch_gram_tc_t(const spod_plan_s& p, const GramTcArgs& a, int grid, size_t smem, cudaStream_t s) {
  auto kern = k_gram_tc<X3, HC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreadsGram, smem, s>>>(p.tmap_hi2, X3 ? p.tmap_lo2 : p.tmap_hi2, a,
                                        reinterpret_cast<uint8_t*>(p.d_gslot), p.d_flags);
  return cudaGetLastError();
}

template <bool X3>
cudaError_t launch_gram_tc_x(const spod_plan_s& p, const GramTcArgs& a, int grid, size_t smem, cudaStream_t s) {
  switch (a.np / 2) {                      // columns per epilogue warp (np is a multiple of 16)
    case 8: return launch_gram_tc_t<X3, 8>(p, a, grid, smem, s);
    case 16: return launch_gram_tc_t<X3, 16>(p, a, grid, smem, s);
    case 24: return launch_gram_tc_t<X3, 24>(p, a, grid, smem, s);
    case 32: return launch_gram_tc_t<X3, 32>(p, a, grid, smem, s);
    case 40: return launch_gram_tc_t<X3, 40>(p, a, grid, smem, s);
    case 48: return launch_gram_tc_t<X3, 48>(p, a, grid, smem, s);
    case 56: return launch_gram_tc_t<X3, 56>(p, a, grid, smem, s);
    case 64: return launch_gram_tc_t<X3, 64>(p, a, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// Shared memory of the smallest (2-stage) configuration; launches use up to 8 stages.
size_t gram_tc_smem_bytes(const spod_plan_s& p) { return gram_tc_smem_stages(p, 2); }

// Slots of the persistent kernel, (max CTAs + nf - 1) x gram_slot_bytes(qrows)
// (counted in doubles), and the per-frequency FP64 accumulator of D over
// chunks, nf x qrows^2 (qrows = 2 nb, + 1 with the folded mean's rho row).
size_t gram_tc_slot_doubles(const spod_plan_s& p, int max_ctas) {
  return ((size_t)(max_ctas + p.nf - 1) * gram_slot_bytes(p.qrows) + 7) / 8;
}
size_t gram_tc_acc_doubles(const spod_plan_s& p) { return (size_t)p.nf * p.qrows * p.qrows; }

// Persistent CTAs of the tensor-core Gram: one per SM unless tuned.
int gram_tc_ctas(const spod_plan_s& p) {
  const int sms = p.num_sms > 0 ? p.num_sms : 148;
  return p.gram_splits > 0 ? std::min(p.gram_splits, p.gram_splits_max) : sms;
}

cudaError_t launch_gram_tc_chunk(const spod_plan_s& p, int64_t mcount, bool first, cudaStream_t s) {
  GramTcArgs a;
  a.nb = p.nb;
  a.r2 = p.qrows;                          // 2 nb, or 2 nb + 1 (rho row, same padding)
  a.np = (2 * p.nb + 15) / 16 * 16;
  a.nf = p.nf;
  a.flush = p.gram_flush > 0 ? p.gram_flush : 1;
  a.box_bytes = (uint32_t)a.np * 128u;
  // A1 buffers: as many as the 512 tensor-memory columns hold beside the two
  // A2 buffers (np = 80 for nb = 38: four), so that short A1 runs are drained
  // while the next ones accumulate
  a.nacc = std::max(2, std::min(kMaxAcc, ((int)kTmemCols - 2 * a.np) / a.np));
  a.stall0 = p.wait_selftest ? 1 : 0;
  a.nblk = (mcount + 63) / 64;
  a.nkb = (a.nblk + kKpb - 1) / kKpb;
  a.nitems = a.nkb * p.nf;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p.device);
  a.nst = kMaxStages;
  while (a.nst > 2 && gram_tc_smem_stages(p, a.nst) > (size_t)optin) --a.nst;
  const size_t smem = gram_tc_smem_stages(p, a.nst);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(gram_tc_ctas(p), a.nitems));
  cudaError_t e = p.desc.precision == SPOD_PREC_BF16X3 ? launch_gram_tc_x<true>(p, a, grid, smem, s)
                                                        : launch_gram_tc_x<false>(p, a, grid, smem, s);
  if (e != cudaSuccess) return e;
  k_gram_tc_collect<<<p.nf, 256, 0, s>>>(reinterpret_cast<const uint8_t*>(p.d_gslot), a.r2, a.nkb, grid,
                                         p.desc.precision == SPOD_PREC_BF16X3 ? 1 : 0, first ? 1 : 0, p.d_gacc);
  return cudaGetLastError();
}

cudaError_t launch_gram_tc_finish(const spod_plan_s& p, cudaStream_t s) {
  k_gram_tc_finish<<<p.nf, 256, 0, s>>>(p.d_gacc, p.nb, p.qrows, p.mean_fold ? p.d_what : nullptr, p.kappa,
                                        p.d_gram, p.d_flags);
  return cudaGetLastError();
}

}  // namespace spod
