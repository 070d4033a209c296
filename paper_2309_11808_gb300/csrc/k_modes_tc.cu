// SPOD modes on the tensor cores (Eq. spod-discrete-snapshots):
// Phi_f[:, k] = Qhat_f psi_k / sqrt(lambda_k / kappa), divided by sqrt(W_m)
// because Qhat carries sqrt(W_m).
//
// Real embedding, per frequency f and tile of 64 points:
//   D[128 x 64] = A[128 x K] * B[64 x K]^T,  K = 2nb (padded to NP = 16 k)
// A (K-major, built once per CTA in shared memory): row k < nmodes holds
// [Re B_f[:, k] ; -Im B_f[:, k]], row nmodes + k holds [Im B_f[:, k] ; Re B_f[:, k]],
// B_f = Psi_f Lambda_f^{-1/2} sqrt(kappa); rows >= 2 nmodes are zero.
// B (MN-major: 64 points contiguous per K row) is the TMA box of Qhat rows,
// the same box the Gram kernel uses.  Then D[k][p] = Re Phi[p][k] and
// D[nmodes + k][p] = Im Phi[p][k].  BF16X3 adds A_hi B_lo + A_lo B_hi.
//
// Warp roles (320 threads): warp 8 issues TMA, warp 9 the MMAs; warps 0-7 drain
// TMEM (double-buffered accumulators; warps w and w+4 share a lane quadrant and
// take one 32-column half each) through shared memory into coalesced complex
// stores of Phi[f][k][m].
#include <algorithm>

#include "tc_common.cuh"

namespace spod {
namespace {

constexpr int kStages = 4;
constexpr uint32_t kTmemCols = 128;       // two 64-column accumulators
constexpr int kPsStride = 65;             // staging row stride (floats): conflict-free rows and columns
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kTmaWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1;
constexpr int kThreadsModes = (kEpiWarps + 2) * 32;

struct ModesTcArgs {
  int nb, nmodes, np, nf;
  int64_t mcount, m0, M, ntiles, tiles_per_cta;
};

struct ModesHdr {
  uint64_t full[kStages], empty[kStages], accfull[2], accempty[2], drain;
  uint32_t tmem_base;
  int abort;
  volatile int decision;
};

__device__ __forceinline__ uint32_t sw128_offset(int r, int kk) {
  // byte offset of BF16 element (row r, k index kk < 64) in a K-major 128-byte-swizzled atom stack
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((kk * 2) >> 4) ^ (r & 7)) << 4) + ((kk * 2) & 15));
}

template <bool X3>
__global__ void __launch_bounds__(kThreadsModes, 1) k_modes_tc(const __grid_constant__ CUtensorMap map_hi,
                                                    const __grid_constant__ CUtensorMap map_lo, ModesTcArgs a,
                                                    const float* __restrict__ bmat, const float* __restrict__ rsqrtW,
                                                    float2* __restrict__ phi, unsigned* __restrict__ gflags) {
  using namespace tc;
  constexpr int NOPS = X3 ? 2 : 1;
  extern __shared__ unsigned char smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  ModesHdr* hdr = reinterpret_cast<ModesHdr*>(sm);
  const int katoms = (a.np + 63) / 64;
  const int a_bytes = katoms * 16384;                      // 128 rows x 64 K per atom
  uint8_t* Ahi = sm + 1024;
  uint8_t* Alo = Ahi + a_bytes;
  const int tile_bytes = ((a.np * 128) + 1023) & ~1023;
  uint8_t* stages = Ahi + NOPS * a_bytes;
  float* Ps = reinterpret_cast<float*>(stages + kStages * NOPS * tile_bytes);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int f = blockIdx.y;
  const int64_t t0 = (int64_t)blockIdx.x * a.tiles_per_cta;
  const int64_t t1 = min(a.ntiles, t0 + a.tiles_per_cta);
  const int ntl = (int)max((int64_t)0, t1 - t0);

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
  // ---- A operand: embedded mode coefficients, BF16 (hi, lo), K-major, 128-byte swizzle
  {
    const int nb = a.nb, nm = a.nmodes;
    const float* Bf = bmat + (size_t)f * nb * nm * 2;
    for (int e = tid; e < 128 * katoms * 64; e += blockDim.x) {
      const int r = e / (katoms * 64);
      const int kap = e - r * (katoms * 64);
      float v = 0.f;
      if (kap < 2 * nb && r < 2 * nm) {
        const int k = r < nm ? r : r - nm;
        const int l = kap < nb ? kap : kap - nb;
        const float br = Bf[(l * nm + k) * 2], bi = Bf[(l * nm + k) * 2 + 1];
        if (r < nm) v = kap < nb ? br : -bi;
        else v = kap < nb ? bi : br;
      }
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      const uint32_t off = (uint32_t)(kap >> 6) * 16384u + sw128_offset(r, kap & 63);
      *reinterpret_cast<__nv_bfloat16*>(Ahi + off) = h;
      if (X3) *reinterpret_cast<__nv_bfloat16*>(Alo + off) = __float2bfloat16_rn(v - __bfloat162float(h));
    }
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = hdr->tmem_base;
  volatile int* abort_flag = &hdr->abort;

  if (warp == kTmaWarp && lane == 0 && ntl > 0) {
    // ---------------- TMA producer
    prefetch_tmap(&map_hi);
    if (X3) prefetch_tmap(&map_lo);
    const uint32_t bytes = (uint32_t)a.np * 128u * NOPS;
    int issued = 0;
    for (int i = 0; i < ntl; ++i) {
      const int s = i % kStages, u = i / kStages;
      if (u >= 1 && !mbar_wait(smem_u32(&hdr->empty[s]), (u - 1) & 1, abort_flag, gflags)) break;
      const uint32_t fb = smem_u32(&hdr->full[s]);
      mbar_arrive_expect_tx(fb, bytes);
      const int kblk = (int)(t0 + i);          // 64-point block of the blocked Qhat layout
      tma_load_4d(smem_u32(stages + (s * NOPS) * tile_bytes), &map_hi, 0, 0, f, kblk, fb);
      if (X3) tma_load_4d(smem_u32(stages + (s * NOPS + 1) * tile_bytes), &map_lo, 0, 0, f, kblk, fb);
      issued = i + 1;
    }
    // copies still in flight must land before the CTA can exit
    for (int i = max(0, issued - kStages); i < issued; ++i)
      mbar_drain(smem_u32(&hdr->full[i % kStages]), (i / kStages) & 1, gflags);
  } else if (warp == kMmaWarp && lane == 0 && ntl > 0) {
    // ---------------- MMA issuer
    const uint32_t idesc = idesc_bf16(128, 64, 0, 1);
    const uint32_t ahi = smem_u32(Ahi), alo = smem_u32(Alo);
    const int nk16 = a.np / 16;
    for (int i = 0; i < ntl; ++i) {
      const int acc = i & 1;
      if (i >= 2 && !mbar_wait(smem_u32(&hdr->accempty[acc]), ((i >> 1) - 1) & 1, abort_flag, gflags)) break;
      const int s = i % kStages, u = i / kStages;
      if (!mbar_wait(smem_u32(&hdr->full[s]), u & 1, abort_flag, gflags)) break;
      tc_fence_after();
      const uint32_t bhi = smem_u32(stages + (s * NOPS) * tile_bytes);
      const uint32_t blo = smem_u32(stages + (s * NOPS + 1) * tile_bytes);
      const uint32_t d = tmem + (uint32_t)acc * 64u;
      for (int j = 0; j < nk16; ++j) {
        const uint32_t aoff = (uint32_t)(j >> 2) * 16384u + (uint32_t)(j & 3) * 32u;
        const uint64_t da = sdesc_sw128(ahi + aoff, 16, 1024);
        const uint64_t db = sdesc_sw128(bhi + (uint32_t)j * 2048u, 1024, 1024);
        mma_bf16(d, da, db, idesc, j > 0 ? 1u : 0u);
        if (X3) {
          const uint64_t dal = sdesc_sw128(alo + aoff, 16, 1024);
          const uint64_t dbl = sdesc_sw128(blo + (uint32_t)j * 2048u, 1024, 1024);
          mma_bf16(d, da, dbl, idesc, 1u);
          mma_bf16(d, dal, db, idesc, 1u);
        }
      }
      mma_commit(smem_u32(&hdr->empty[s]));
      mma_commit(smem_u32(&hdr->accfull[acc]));
    }
    mma_commit(smem_u32(&hdr->drain));
    mbar_drain(smem_u32(&hdr->drain), 0, gflags);
  } else if (warp < kEpiWarps) {
    // ---------------- epilogue
    const int row = (warp & 3) * 32 + lane;
    const int half = warp >> 2;               // columns [32 half, 32 half + 32)
    const int nm = a.nmodes;
    const int jpt = tid & 63, k0 = tid >> 6;  // output: point jpt, modes k0, k0 + 4, ...
    for (int i = 0; i < ntl; ++i) {
      const int acc = i & 1;
      // every epilogue thread takes the same stop/continue decision, so none
      // can be left behind in a named barrier
      mbar_wait(smem_u32(&hdr->accfull[acc]), (i >> 1) & 1, abort_flag, gflags);
      named_sync(1, kEpiThreads);
      if (tid == 0) hdr->decision = *abort_flag;
      named_sync(1, kEpiThreads);
      if (hdr->decision) break;
      tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)acc * 64u + 32u * half;
      {
        float v[32], w[32];
        tmem_ld32x2(taddr, taddr, v, w);           // this warp's 32 columns, one wait
        if (row < 2 * nm) {
#pragma unroll
          for (int q = 0; q < 32; ++q) Ps[row * kPsStride + 32 * half + q] = v[q];
        }
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&hdr->accempty[acc]));
      named_sync(1, kEpiThreads);
      const int64_t lm = (t0 + i) * 64 + jpt;
      if (lm < a.mcount) {
        const int64_t m = a.m0 + lm;
        const float rw = rsqrtW[m];
        for (int k = k0; k < nm; k += kEpiThreads / 64) {
          float2 o;
          o.x = Ps[k * kPsStride + jpt] * rw;
          o.y = Ps[(nm + k) * kPsStride + jpt] * rw;
          phi[((int64_t)f * nm + k) * a.M + m] = o;
        }
      }
      named_sync(1, kEpiThreads);
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

size_t modes_tc_smem_bytes(const spod_plan_s& p) {
  const int nops = p.desc.precision == SPOD_PREC_BF16X3 ? 2 : 1;
  const int np = (2 * p.nb + 15) / 16 * 16;
  const int katoms = (np + 63) / 64;
  const size_t tile_bytes = ((size_t)(np * 128) + 1023) & ~size_t(1023);
  return 1024 + 1024 + (size_t)nops * katoms * 16384 + (size_t)kStages * nops * tile_bytes +
         sizeof(float) * 128 * kPsStride;
}

cudaError_t launch_modes_tc_chunk(const spod_plan_s& p, int64_t m0, int64_t mcount, int nmodes, void* d_Phi,
                                  cudaStream_t s, bool adjoint) {
  const float* scale = static_cast<const float*>(adjoint ? p.d_sqrtW : p.d_rsqrtW);
  ModesTcArgs a;
  a.nb = p.nb;
  a.nmodes = nmodes;
  a.np = (2 * p.nb + 15) / 16 * 16;
  a.nf = p.nf;
  a.mcount = mcount;
  a.m0 = m0;
  a.M = p.M;
  a.ntiles = (mcount + 63) / 64;
  const int sms = p.num_sms > 0 ? p.num_sms : 148;
  int g = 1;
  double best = 1e30;
  for (int c = 1; c <= 64 && c <= a.ntiles; ++c) {
    const int64_t ctas = (int64_t)c * p.nf;
    const int64_t waves = (ctas + sms - 1) / sms;
    const double waste = (double)(waves * sms - ctas) / (double)ctas + (waves < 4 ? 1.0 : 0.0);
    if (waste < best - 1e-9) { best = waste; g = c; }
  }
  if (p.modes_ctas > 0) g = (int)std::min<int64_t>(p.modes_ctas, a.ntiles);
  a.tiles_per_cta = (a.ntiles + g - 1) / g;
  const int gx = (int)((a.ntiles + a.tiles_per_cta - 1) / a.tiles_per_cta);
  const size_t smem = modes_tc_smem_bytes(p);
  dim3 grid((unsigned)gx, (unsigned)p.nf);
  if (p.desc.precision == SPOD_PREC_BF16X3) {
    cudaError_t e = cudaFuncSetAttribute(k_modes_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_modes_tc<true><<<grid, kThreadsModes, smem, s>>>(p.tmap_hi, p.tmap_lo, a, static_cast<const float*>(p.d_bmat),
                                             scale, static_cast<float2*>(d_Phi), p.d_flags);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_modes_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_modes_tc<false><<<grid, kThreadsModes, smem, s>>>(p.tmap_hi, p.tmap_hi, a, static_cast<const float*>(p.d_bmat),
                                              scale, static_cast<float2*>(d_Phi), p.d_flags);
  }
  return cudaGetLastError();
}

}  // namespace spod
