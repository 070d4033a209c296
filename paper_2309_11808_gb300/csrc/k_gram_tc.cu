// Weighted Gram on the 5th-generation tensor cores (Eq. spod-discrete-snapshots):
// M_f = kappa * Qhat_f^* W Qhat_f from BF16 operands (BF16 precision) or from
// the split x = hi + lo (BF16X3 precision), FP32 accumulation in tensor memory.
//
// BF16X3 uses three MMAs per K step and still keeps all four product terms:
// the Gram is symmetric, so with A1 = Yhi Yhi^T + Ylo Ylo^T and A2 = Yhi Ylo^T
// (two TMEM accumulators), Y Y^T = A1 + A2 + A2^T.  Dropping Ylo Ylo^T instead
// would bias the diagonal low by E[lo^2] / x^2 ~ 2.4e-6 and move small
// eigenvalues by that much times (tr M_f / nb) / lambda_k.
//
// Real embedding: with Y_f = [Re Qhat_f ; Im Qhat_f] (2nb rows x points, K-major
// in HBM), D = Y_f Y_f^T gives
//   Re M_f[l][l'] = D[l][l'] + D[nb+l][nb+l'],  Im M_f[l][l'] = D[l][nb+l'] - D[nb+l][l'].
// One TMA box (64 points x NP rows, NP = 2nb rounded up to 16, 128-byte
// swizzle) is both the A operand (M = 128 rows; rows >= NP are zero) and the
// B operand (N = NP) of tcgen05.mma.cta_group::1.kind::f16, K = 16 per
// instruction, 4 instructions per 64-point block (x3 for BF16X3).
//
// Warp roles (320 threads): warp 8 lane 0 issues TMA into a 4-stage ring,
// warp 9 lane 0 issues the MMAs, warps 0-7 (two per TMEM lane quadrant) drain
// the accumulators every `flush` blocks of 64 points (short FP32 runs in the
// tensor core) and add them into compensated FP32 (sum, carry) registers.
// The accumulators are double-buffered in TMEM so draining overlaps the next
// group's MMAs; the drain stages S1 = A1 + A2 and S2 = A2 in shared memory
// (Y Y^T = S1 + S2^T) with one TMEM wait per 32 columns.  Partials per (split, frequency) go to the same FP64 buffer as
// the SIMT kernel and are reduced in fixed order by k_gram_reduce.
#include "tc_common.cuh"

namespace spod {
namespace {

constexpr int kStages = 4;
constexpr int kTileBytes = 128 * 128;     // 128 rows x 64 BF16
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kTmaWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1;
constexpr int kThreadsGram = (kEpiWarps + 2) * 32;
constexpr int kMaxPerThread = 9;          // nb <= 64: nb (nb+1) / 2 <= 9 * 256
constexpr uint32_t kTmemCols = 512;       // buffer b: A1 at 256 b, A2 at 256 b + 128

struct GramTcArgs {
  int nb, rows2, np, nf, ne;
  int64_t kb_per_split, nkb;              // 64-point blocks per split, blocks in the chunk
  int first;
  int flush;                              // blocks per FP32 accumulation group
};

// Neumaier compensated addition: (s, c) += y
__device__ __forceinline__ void comp_add(float& s, float& c, float y) {
  const float t = s + y;
  c += fabsf(s) >= fabsf(y) ? (s - t) + y : (y - t) + s;
  s = t;
}

struct GramHdr {
  uint64_t full[kStages], empty[kStages], accfull[2], accempty[2], drain;
  uint32_t tmem_base;
  int abort;
  volatile int decision;
};

template <bool X3>
__global__ void __launch_bounds__(kThreadsGram, 1) k_gram_tc(const __grid_constant__ CUtensorMap map_hi,
                                                   const __grid_constant__ CUtensorMap map_lo, GramTcArgs a,
                                                   double* __restrict__ gpart, unsigned* __restrict__ gflags) {
  using namespace tc;
  constexpr int NOPS = X3 ? 2 : 1;
  extern __shared__ unsigned char smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  GramHdr* hdr = reinterpret_cast<GramHdr*>(sm);
  uint8_t* stages = sm + 1024;
  const int RS = a.rows2 | 1;               // odd staging stride: conflict-free rows and columns
  float* Ds = reinterpret_cast<float*>(stages + kStages * NOPS * kTileBytes);   // S1 = A1 + A2
  float* Qs = Ds + a.rows2 * RS;                                                  // S2 = A2 (BF16X3)
  uint32_t* pairs = reinterpret_cast<uint32_t*>(Qs + (X3 ? a.rows2 * RS : 0));

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s_idx = blockIdx.x, f = blockIdx.y;
  const int64_t kb0 = (int64_t)s_idx * a.kb_per_split;
  const int64_t kb1 = min(a.nkb, kb0 + a.kb_per_split);
  const int nkbl = (int)max((int64_t)0, kb1 - kb0);
  const int FB = a.flush;
  const int ngroups = (nkbl + FB - 1) / FB;

  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(smem_u32(&hdr->full[i]), 1);
      mbar_init(smem_u32(&hdr->empty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&hdr->accfull[i]), 1);
      mbar_init(smem_u32(&hdr->accempty[i]), kEpiThreads);
    }
    mbar_init(smem_u32(&hdr->drain), 1);
    hdr->abort = 0;
    fence_mbar_init();
  }
  if (warp == kMmaWarp) {
    tmem_alloc(smem_u32(&hdr->tmem_base), kTmemCols);
    tmem_relinquish();
  }
  // rows np..127 of every stage tile are never written by TMA: zero them once
  {
    const int pad_bytes = (128 - a.np) * 128;
    for (int t = 0; t < kStages * NOPS; ++t) {
      uint4* p = reinterpret_cast<uint4*>(stages + t * kTileBytes + a.np * 128);
      for (int i = tid; i < pad_bytes / 16; i += blockDim.x) p[i] = make_uint4(0, 0, 0, 0);
    }
  }
  for (int e = tid; e < a.ne; e += blockDim.x) {
    // e -> (l, l'), l <= l', row-major over the upper triangle
    int l = 0, rem = e;
    while (rem >= a.nb - l) { rem -= a.nb - l; ++l; }
    pairs[e] = (uint32_t)l | ((uint32_t)(l + rem) << 16);
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = hdr->tmem_base;
  volatile int* abort_flag = &hdr->abort;

  if (warp == kTmaWarp && lane == 0 && nkbl > 0) {
    // ---------------- TMA producer
    prefetch_tmap(&map_hi);
    if (X3) prefetch_tmap(&map_lo);
    const uint32_t bytes = (uint32_t)a.np * 128u * NOPS;
    int issued = 0;
    for (int kb = 0; kb < nkbl; ++kb) {
      const int s = kb % kStages, u = kb / kStages;
      if (u >= 1 && !mbar_wait(smem_u32(&hdr->empty[s]), (u - 1) & 1, abort_flag, gflags)) break;
      const uint32_t fb = smem_u32(&hdr->full[s]);
      mbar_arrive_expect_tx(fb, bytes);
      const int kblk = (int)(kb0 + kb);        // 64-point block of the blocked Qhat layout
      tma_load_4d(smem_u32(stages + (s * NOPS) * kTileBytes), &map_hi, 0, 0, f, kblk, fb);
      if (X3) tma_load_4d(smem_u32(stages + (s * NOPS + 1) * kTileBytes), &map_lo, 0, 0, f, kblk, fb);
      issued = kb + 1;
    }
    // copies still in flight must land before the CTA can exit
    for (int kb = max(0, issued - kStages); kb < issued; ++kb)
      mbar_drain(smem_u32(&hdr->full[kb % kStages]), (kb / kStages) & 1, gflags);
  } else if (warp == kMmaWarp && lane == 0 && nkbl > 0) {
    // ---------------- MMA issuer
    const uint32_t idesc = idesc_bf16(128, a.np, 0, 0);
    for (int kb = 0; kb < nkbl; ++kb) {
      const int g = kb / FB, acc = g & 1;
      const bool gfirst = (kb % FB) == 0;
      if (gfirst && g >= 2 && !mbar_wait(smem_u32(&hdr->accempty[acc]), ((g >> 1) - 1) & 1, abort_flag, gflags))
        break;
      const int s = kb % kStages, u = kb / kStages;
      if (!mbar_wait(smem_u32(&hdr->full[s]), u & 1, abort_flag, gflags)) break;
      tc_fence_after();
      const uint32_t hi = smem_u32(stages + (s * NOPS) * kTileBytes);
      const uint32_t lo = smem_u32(stages + (s * NOPS + 1) * kTileBytes);
      const uint32_t d1 = tmem + (uint32_t)acc * 256u;
      const uint32_t d2 = d1 + 128u;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t first_k = (gfirst && k == 0) ? 0u : 1u;
        const uint64_t dh = sdesc_sw128(hi + k * 32, 16, 1024);
        mma_bf16(d1, dh, dh, idesc, first_k);
        if (X3) {
          const uint64_t dl = sdesc_sw128(lo + k * 32, 16, 1024);
          mma_bf16(d1, dl, dl, idesc, 1u);
          mma_bf16(d2, dh, dl, idesc, first_k);
        }
      }
      mma_commit(smem_u32(&hdr->empty[s]));
      if ((kb % FB) == FB - 1 || kb == nkbl - 1) mma_commit(smem_u32(&hdr->accfull[acc]));
    }
    mma_commit(smem_u32(&hdr->drain));
    mbar_drain(smem_u32(&hdr->drain), 0, gflags);
  } else if (warp < kEpiWarps) {
    // ---------------- epilogue: TMEM -> FP32 staging -> compensated FP32 sums
    float sr[kMaxPerThread], cr[kMaxPerThread], si[kMaxPerThread], ci[kMaxPerThread];
#pragma unroll
    for (int j = 0; j < kMaxPerThread; ++j) { sr[j] = 0.f; cr[j] = 0.f; si[j] = 0.f; ci[j] = 0.f; }
    const int row = (warp & 3) * 32 + lane;
    const int half = warp >> 2;               // takes the 32-column chunks c0 = 32 (2 k + half)
    const int nb = a.nb, r2 = a.rows2;
    for (int g = 0; g < ngroups; ++g) {
      const int acc = g & 1;
      // every epilogue thread takes the same stop/continue decision, so none
      // can be left behind in a named barrier
      mbar_wait(smem_u32(&hdr->accfull[acc]), (g >> 1) & 1, abort_flag, gflags);
      named_sync(1, kEpiThreads);
      if (tid == 0) hdr->decision = *abort_flag;
      named_sync(1, kEpiThreads);
      if (hdr->decision) break;
      tc_fence_after();
      const uint32_t t1 = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)acc * 256u;
      // stage S1 = A1 + A2 and S2 = A2 row by row (D = S1 + S2^T); 32 columns of
      // each accumulator per load batch, one wait per batch
      for (int c0 = 32 * half; c0 < a.np; c0 += 64) {
        float v[32], w[32];
        if (X3) {
          tmem_ld32x2(t1 + c0, t1 + 128 + c0, v, w);
        } else {
          tmem_ld32x2(t1 + c0, t1 + c0, v, w);
        }
        if (row < r2) {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            if (c0 + i < r2) {
              Ds[row * RS + c0 + i] = X3 ? v[i] + w[i] : v[i];
              if (X3) Qs[row * RS + c0 + i] = w[i];
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&hdr->accempty[acc]));
      named_sync(1, kEpiThreads);
#pragma unroll
      for (int j = 0; j < kMaxPerThread; ++j) {
        const int e = tid + kEpiThreads * j;
        if (e < a.ne) {
          const uint32_t pr = pairs[e];
          const int l = pr & 0xFFFF, lp = pr >> 16;
          // D[i][k] = S1[i][k] + S2[k][i]
          float d1 = Ds[l * RS + lp] + Ds[(nb + l) * RS + nb + lp];
          float d2 = Ds[l * RS + nb + lp] - Ds[(nb + l) * RS + lp];
          if (X3) {
            d1 += Qs[lp * RS + l] + Qs[(nb + lp) * RS + nb + l];
            d2 += Qs[(nb + lp) * RS + l] - Qs[lp * RS + nb + l];
          }
          comp_add(sr[j], cr[j], d1);
          comp_add(si[j], ci[j], d2);
        }
      }
      named_sync(1, kEpiThreads);
    }
    double* gp = gpart + (((int64_t)s_idx * a.nf + f) * nb) * nb * 2;
#pragma unroll
    for (int j = 0; j < kMaxPerThread; ++j) {
      const int e = tid + kEpiThreads * j;
      if (e < a.ne) {
        const uint32_t pr = pairs[e];
        const int l = pr & 0xFFFF, lp = pr >> 16;
        double* o = gp + ((int64_t)l * nb + lp) * 2;
        const double vr = (double)sr[j] + (double)cr[j], vi = (double)si[j] + (double)ci[j];
        if (a.first) { o[0] = vr; o[1] = vi; }
        else { o[0] += vr; o[1] += vi; }
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

}  // namespace

size_t gram_tc_smem_bytes(const spod_plan_s& p) {
  const int nops = p.desc.precision == SPOD_PREC_BF16X3 ? 2 : 1;
  const int r2 = 2 * p.nb;
  const int ne = p.nb * (p.nb + 1) / 2;
  return 1024 + 1024 + (size_t)kStages * nops * kTileBytes + sizeof(float) * r2 * (r2 | 1) * nops +
         sizeof(uint32_t) * ne;
}

int gram_tc_splits(const spod_plan_s& p, int64_t nkb) {
  // splits per frequency: at least 8 waves of one CTA per SM, least tail
  const int sms = p.num_sms > 0 ? p.num_sms : 148;
  int best = 1;
  double best_waste = 1e30;
  for (int s = 1; s <= 32; ++s) {
    if (s > nkb) break;
    const int64_t ctas = (int64_t)s * p.nf;
    const int64_t waves = (ctas + sms - 1) / sms;
    const double waste = (double)(waves * sms - ctas) / (double)ctas + (waves < 4 ? 1.0 : 0.0);
    if (waste < best_waste - 1e-9) { best_waste = waste; best = s; }
  }
  return best;
}

cudaError_t launch_gram_tc_chunk(const spod_plan_s& p, int64_t mcount, bool first, cudaStream_t s) {
  GramTcArgs a;
  a.nb = p.nb;
  a.rows2 = 2 * p.nb;
  a.np = (2 * p.nb + 15) / 16 * 16;
  a.nf = p.nf;
  a.ne = p.nb * (p.nb + 1) / 2;
  a.nkb = (mcount + 63) / 64;
  const int splits = p.gram_splits;
  a.kb_per_split = (a.nkb + splits - 1) / splits;
  a.first = first ? 1 : 0;
  a.flush = p.gram_flush > 0 ? p.gram_flush : 4;
  const size_t smem = gram_tc_smem_bytes(p);
  dim3 grid((unsigned)splits, (unsigned)p.nf);
  if (p.desc.precision == SPOD_PREC_BF16X3) {
    cudaError_t e = cudaFuncSetAttribute(k_gram_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gram_tc<true><<<grid, kThreadsGram, smem, s>>>(p.tmap_hi, p.tmap_lo, a, p.d_gpart, p.d_flags);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_gram_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gram_tc<false><<<grid, kThreadsGram, smem, s>>>(p.tmap_hi, p.tmap_hi, a, p.d_gpart, p.d_flags);
  }
  return cudaGetLastError();
}

}  // namespace spod
