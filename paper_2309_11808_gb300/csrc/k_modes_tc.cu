// SPOD modes on the tensor cores (Eq. spod-discrete-snapshots):
// Phi_f[:, k] = Qhat_f psi_k / sqrt(lambda_k / kappa), divided by sqrt(W_m)
// because Qhat carries sqrt(W_m).
//
// Real embedding, per frequency f and tile of 128 points (two 64-point blocks
// of the blocked Qhat layout):
//   D[128 points x NN] = A[128 x K] * B[NN x K]^T,  K = 2 nb (padded to 16)
// A is MN-major: the two TMA boxes of Qhat (K rows x 64 points each) side by
// side.  B (K-major, 128-byte swizzle) is a per-frequency image built once per
// call in global memory (k_mode_image) and copied into shared memory by one
// bulk copy whenever a CTA moves to the next frequency: row 2k holds
// [Re B_f[:, k] ; -Im B_f[:, k]], row 2k+1 holds [Im B_f[:, k] ; Re B_f[:, k]],
// B_f = Psi_f Lambda_f^{-1/2} sqrt(kappa), so D[p][2k] = Re Phi[p][k] and
// D[p][2k+1] = Im Phi[p][k]: each TMEM lane (one point) holds interleaved
// complex outputs, stored straight from registers as 8-byte values, 256
// contiguous bytes per warp and mode.  BF16X3 adds A_hi B_lo + A_lo B_hi.
// With B = G_f and scale sqrt(W) the same kernel computes W Qhat G_f for the
// adjoint.
//
// Persistent CTAs (one per SM) walk a contiguous range of the f-major list of
// (frequency, 128-point tile) items.  Warp roles (320 threads): warp 8 issues
// TMA (and the B image copy at each frequency change), warp 9 issues the MMAs
// into two TMEM accumulators, warps 0-7 drain them (warps w and w+4 share a
// lane quadrant and take one half of the columns each).  Every wait is bounded.
#include <algorithm>

#include "tc_common.cuh"

namespace spod {
namespace {

constexpr int kMaxStages = 4;            // pipeline depth (fewer when shared memory is short)
constexpr int kMaxImageModes = 128;      // modes of one image (nmodes <= nb; the tensor path keeps 2 nb <= 128)
constexpr uint32_t kTmemCols = 256;       // two accumulators at columns 0 and 128
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kTmaWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1;
constexpr int kThreadsModes = (kEpiWarps + 2) * 32;

struct ModesTcArgs {
  int nb, nmodes, np, nn, nf;             // np = K (2 nb padded to 16), nn = N (2 nmodes padded to 16)
  int64_t mcount, m0, M;                  // M: row stride of Phi in points
  int64_t phioff;                          // point of Phi's first column (tiled output)
  int64_t ntp;                             // 128-point tiles per frequency
  int64_t qtile0;                          // first 128-point tile of the call inside the Qhat chunk
  int64_t nitems;                          // (f1 - f0) * ntp
  int f0;                                  // first frequency of the call's range
  uint32_t box_bytes;                      // one Qhat TMA box: np rows x 128 bytes
  uint32_t img_bytes;                      // one B image (hi or lo)
  int nst;                                 // pipeline stages (2 .. kMaxStages)
};

struct ModesHdr {
  uint64_t full[kMaxStages], empty[kMaxStages], accfull[2], accempty[2], bfull, bempty, drain;
  uint32_t tmem_base;
  int abort;
};

__device__ __forceinline__ uint32_t sw128_offset(int r, int kk) {
  // byte offset of BF16 element (row r, k index kk < 64) in a K-major 128-byte-swizzled atom stack
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((kk * 2) >> 4) ^ (r & 7)) << 4) + ((kk * 2) & 15));
}

// 1-D bulk copy global -> shared with mbarrier completion (16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
               : "memory");
}

// 8 consecutive TMEM columns of this thread's lane (no wait).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// B image of frequency f: rows n < nn (2k: real part of mode k, 2k+1: imaginary
// part), K index kk < np (l: Re Qhat row l, nb + l: Im Qhat row l), BF16 hi
// (and lo = bf16(v - hi)), K-major 128-byte-swizzled atoms of 64 K values.
__global__ void k_mode_image(const float* __restrict__ bmat, int nb, int nm, int np, int nn, int x3,
                             const double* __restrict__ what, uint32_t img_bytes, uint8_t* __restrict__ img) {
  const int f = blockIdx.x;
  const float* Bf = bmat + (size_t)f * nb * nm * 2;
  // folded mean: the correction row's entries -What_f c_k, c_k = sum_l B_f[l][k],
  // one thread per mode (FP64 sums of the FP32 coefficients), before the image loop
  __shared__ float2 corr[kMaxImageModes];
  if (what) {
    const double wr = what[2 * f], wi = what[2 * f + 1];
    for (int k = threadIdx.x; k < nm; k += blockDim.x) {
      double cr = 0.0, ci = 0.0;
      for (int l = 0; l < nb; ++l) {
        cr += (double)Bf[(l * nm + k) * 2];
        ci += (double)Bf[(l * nm + k) * 2 + 1];
      }
      corr[k] = make_float2((float)-(wr * cr - wi * ci), (float)-(wr * ci + wi * cr));
    }
    __syncthreads();
  }
  uint8_t* hi = img + (size_t)f * img_bytes * (x3 ? 2 : 1);
  uint8_t* lo = hi + img_bytes;
  const int katoms = (np + 63) / 64;
  for (int e = threadIdx.x; e < nn * katoms * 64; e += blockDim.x) {
    const int n = e / (katoms * 64);
    const int kk = e - n * (katoms * 64);
    const int k = n >> 1;
    float v = 0.f;
    if (kk < 2 * nb && k < nm) {
      const int l = kk < nb ? kk : kk - nb;
      const float br = Bf[(l * nm + k) * 2], bi = Bf[(l * nm + k) * 2 + 1];
      if ((n & 1) == 0) v = kk < nb ? br : -bi;
      else v = kk < nb ? bi : br;
    } else if (what && kk == 2 * nb && k < nm) {
      // folded mean: Qhat rows are the spectra Z of x - c, row 2 nb is rho; the
      // spectra of x - mu are Z - rho What_f, so column k gains -rho What_f c_k
      v = (n & 1) == 0 ? corr[k].x : corr[k].y;
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const uint32_t off = (uint32_t)(kk >> 6) * (uint32_t)(nn * 128) + sw128_offset(n, kk & 63);
    *reinterpret_cast<__nv_bfloat16*>(hi + off) = h;
    if (x3) *reinterpret_cast<__nv_bfloat16*>(lo + off) = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// Position of a CTA's item in the (frequency, tile) list and in the stage
// ring, advanced without divisions (the issuing threads are on the critical
// path of every item).
struct Cursor {
  int f, tp;          // frequency, 128-point tile within it
  int s, ph;          // stage, parity of the ring pass (i / nst) & 1
  __device__ __forceinline__ void init(int64_t item0, int ntp, int f0) {
    const int fr = (int)(item0 / ntp);
    tp = (int)(item0 - (int64_t)fr * ntp);
    f = f0 + fr;
    s = 0;
    ph = 0;
  }
  __device__ __forceinline__ void next(int ntp, int nst) {
    if (++tp == ntp) { tp = 0; ++f; }
    if (++s == nst) { s = 0; ph ^= 1; }
  }
};

template <bool X3>
__global__ void __launch_bounds__(kThreadsModes, 1) k_modes_tc(const __grid_constant__ CUtensorMap map_hi,
                                                    const __grid_constant__ CUtensorMap map_lo, ModesTcArgs a,
                                                    const uint8_t* __restrict__ img, const float* __restrict__ scale,
                                                    float2* __restrict__ phi, unsigned* __restrict__ gflags) {
  using namespace tc;
  constexpr int NOPS = X3 ? 2 : 1;
  extern __shared__ unsigned char smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  ModesHdr* hdr = reinterpret_cast<ModesHdr*>(sm);
  uint8_t* Bhi = sm + 1024;
  uint8_t* Blo = Bhi + a.img_bytes;
  const uint32_t stage_bytes = 2u * a.box_bytes * NOPS;   // two 64-point boxes (hi [, lo])
  uint8_t* stages = Bhi + NOPS * a.img_bytes;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t i0 = a.nitems * blockIdx.x / gridDim.x;
  const int64_t i1 = a.nitems * (blockIdx.x + 1) / gridDim.x;
  const int nit = (int)(i1 - i0);
  const int ntp = (int)a.ntp;

  if (tid == 0) {
    for (int i = 0; i < a.nst; ++i) {
      mbar_init(smem_u32(&hdr->full[i]), 1);
      mbar_init(smem_u32(&hdr->empty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&hdr->accfull[i]), 1);
      mbar_init(smem_u32(&hdr->accempty[i]), kEpiThreads);
    }
    mbar_init(smem_u32(&hdr->bfull), 1);
    mbar_init(smem_u32(&hdr->bempty), 1);
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
    // ---------------- TMA producer (+ B image at each frequency change)
    prefetch_tmap(&map_hi);
    if (X3) prefetch_tmap(&map_lo);
    int issued = 0, seg = 0, segs_loaded = 0;
    int fcur = -1;
    Cursor cu;
    cu.init(i0, ntp, a.f0);
    for (int i = 0; i < nit; ++i, cu.next(ntp, a.nst)) {
      const int f = cu.f, tp = cu.tp;
      if (f != fcur) {
        // the MMAs of the previous frequency must be done with B before it is replaced
        if (seg >= 1 && !mbar_wait(smem_u32(&hdr->bempty), (seg - 1) & 1, abort_flag, gflags)) break;
        const uint32_t bb = smem_u32(&hdr->bfull);
        mbar_arrive_expect_tx(bb, a.img_bytes * NOPS);
        const uint8_t* src = img + (size_t)f * a.img_bytes * NOPS;
        bulk_load(smem_u32(Bhi), src, a.img_bytes, bb);
        if (X3) bulk_load(smem_u32(Blo), src + a.img_bytes, a.img_bytes, bb);
        segs_loaded = seg + 1;
        fcur = f;
        ++seg;
      }
      const int s = cu.s;
      if (i >= a.nst && !mbar_wait(smem_u32(&hdr->empty[s]), cu.ph ^ 1, abort_flag, gflags)) break;
      const uint32_t fb = smem_u32(&hdr->full[s]);
      mbar_arrive_expect_tx(fb, stage_bytes);
      uint8_t* st = stages + (size_t)s * stage_bytes;
      const int kb = 2 * (tp + (int)a.qtile0);
      // one copy per operand: the tile's two 64-point blocks side by side
      tma_load_4d(smem_u32(st), &map_hi, 0, 0, f, kb, fb);
      if (X3) tma_load_4d(smem_u32(st + 2 * a.box_bytes), &map_lo, 0, 0, f, kb, fb);
      issued = i + 1;
    }
    // copies still in flight must land before the CTA can exit
    for (int i = max(0, issued - a.nst); i < issued; ++i)
      mbar_drain(smem_u32(&hdr->full[i % a.nst]), (i / a.nst) & 1, gflags);
    if (segs_loaded > 0) mbar_drain(smem_u32(&hdr->bfull), (segs_loaded - 1) & 1, gflags);
  } else if (warp == kMmaWarp && lane == 0 && nit > 0) {
    // ---------------- MMA issuer
    const uint32_t idesc = idesc_bf16(128, a.nn, 1, 0);      // A MN-major (points), B K-major
    const uint32_t bhi = smem_u32(Bhi), blo = smem_u32(Blo);
    const uint32_t katom_bytes = (uint32_t)a.nn * 128u;
    const int nk16 = a.np / 16;
    int seg = 0;
    int fcur = -1;
    Cursor cu;
    cu.init(i0, ntp, a.f0);
    for (int i = 0; i < nit; ++i, cu.next(ntp, a.nst)) {
      const int f = cu.f;
      if (f != fcur) {
        if (seg >= 1) mma_commit(smem_u32(&hdr->bempty));   // B of the previous frequency is released
        if (!mbar_wait(smem_u32(&hdr->bfull), seg & 1, abort_flag, gflags)) break;
        fcur = f;
        ++seg;
      }
      const int acc = i & 1;
      if (i >= 2 && !mbar_wait(smem_u32(&hdr->accempty[acc]), ((i >> 1) - 1) & 1, abort_flag, gflags)) break;
      const int s = cu.s;
      if (!mbar_wait(smem_u32(&hdr->full[s]), cu.ph, abort_flag, gflags)) break;
      tc_fence_after();
      const uint32_t st = smem_u32(stages + (size_t)s * stage_bytes);
      const uint32_t d = tmem + (uint32_t)acc * 128u;
      for (int j = 0; j < nk16; ++j) {
        // A: 16 K rows of both point boxes (MN atoms box_bytes apart); B: 16 K columns
        const uint64_t da = sdesc_sw128(st + (uint32_t)j * 2048u, a.box_bytes, 1024);
        const uint32_t boff = (uint32_t)(j >> 2) * katom_bytes + (uint32_t)(j & 3) * 32u;
        const uint64_t db = sdesc_sw128(bhi + boff, 16, 1024);
        mma_bf16(d, da, db, idesc, j > 0 ? 1u : 0u);
        if (X3) {
          const uint64_t dal = sdesc_sw128(st + 2 * a.box_bytes + (uint32_t)j * 2048u, a.box_bytes, 1024);
          const uint64_t dbl = sdesc_sw128(blo + boff, 16, 1024);
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
    // ---------------- epilogue: TMEM -> registers -> scaled complex stores
    const int quad = warp & 3;
    const int half = warp >> 2;
    const int hcols = a.nn / 2;                     // columns of this warp: [half * hcols, +hcols)
    const int k0 = half * (hcols / 2);              // first mode of this warp
    const int nm = a.nmodes;
    Cursor cu;
    cu.init(i0, ntp, a.f0);
    for (int i = 0; i < nit; ++i, cu.next(ntp, a.nst)) {
      const int f = cu.f, tp = cu.tp;
      const int acc = i & 1;
      // the point's output scale, requested before the wait for the
      // accumulator so that its latency overlaps the item's copies and MMAs
      const int64_t lm = tp * 128 + quad * 32 + lane;
      const bool inrange = lm < a.mcount;
      const float rw = inrange ? scale[a.m0 + lm] : 0.f;
      // one decision per warp: the tcgen05.ld below must be executed by the whole warp
      const bool got = mbar_wait(smem_u32(&hdr->accfull[acc]), (i >> 1) & 1, abort_flag, gflags);
      if (!__all_sync(0xffffffffu, got)) break;
      tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)acc * 128u + (uint32_t)(half * hcols);
      float v[64];
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (c * 8 < hcols) tmem_ld8(taddr + (uint32_t)(c * 8), v + c * 8);
      tmem_wait_ld();
      tc_fence_before();
      mbar_arrive(smem_u32(&hdr->accempty[acc]));
      if (inrange) {
        const int64_t m = a.m0 + lm;
        float2* out = phi + ((int64_t)f * nm + k0) * a.M + (m - a.phioff);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (2 * j < hcols && k0 + j < nm) out[(int64_t)j * a.M] = make_float2(v[2 * j] * rw, v[2 * j + 1] * rw);
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

int modes_np(const spod_plan_s& p) { return (2 * p.nb + 15) / 16 * 16; }
int modes_nn(int nmodes) { return (2 * nmodes + 15) / 16 * 16; }
uint32_t modes_img_bytes(int np, int nn) { return (uint32_t)((np + 63) / 64) * (uint32_t)nn * 128u; }

size_t modes_tc_smem_stages(const spod_plan_s& p, int nst) {
  const int nops = p.desc.precision == SPOD_PREC_BF16X3 ? 2 : 1;
  const int np = modes_np(p);
  const size_t img = modes_img_bytes(np, modes_nn(std::max(p.nb, p.adj_cols)));   // the adjoint's extra column
  const size_t box = (size_t)np * 128;
  return 1024 + 1024 + nops * img + (size_t)nst * 2 * box * nops;
}

}  // namespace

// Shared memory of the smallest (2-stage) configuration; launches use up to 4 stages.
size_t modes_tc_smem_bytes(const spod_plan_s& p) { return modes_tc_smem_stages(p, 2); }

// Per-frequency B images (hi [, lo]) for nmodes columns, in the plan's image buffer.
size_t modes_image_bytes(const spod_plan_s& p) {
  const int nops = p.desc.precision == SPOD_PREC_BF16X3 ? 2 : 1;
  return (size_t)p.nf * nops * modes_img_bytes(modes_np(p), modes_nn(std::max(p.nb, p.adj_cols)));
}

cudaError_t launch_mode_image(const spod_plan_s& p, int nmodes, cudaStream_t s) {
  const int np = modes_np(p), nn = modes_nn(nmodes);
  if (nmodes > kMaxImageModes) return cudaErrorInvalidValue;
  k_mode_image<<<p.nf, 256, 0, s>>>(static_cast<const float*>(p.d_bmat), p.nb, nmodes, np, nn,
                                    p.desc.precision == SPOD_PREC_BF16X3 ? 1 : 0,
                                    p.mean_fold ? p.d_what : nullptr, modes_img_bytes(np, nn),
                                    static_cast<uint8_t*>(p.d_bimg));
  return cudaGetLastError();
}

cudaError_t launch_modes_tc_chunk(const spod_plan_s& p, int64_t m0, int64_t mcount, int nmodes, void* d_Phi,
                                  cudaStream_t s, bool adjoint, int f0, int f1, int64_t qoff, int64_t out_ld,
                                  int64_t out_off) {
  if (qoff % 128 != 0) return cudaErrorInvalidValue;
  if (f1 < 0) f1 = p.nf;
  if (f0 < 0 || f1 > p.nf || f0 >= f1) return cudaErrorInvalidValue;
  const float* scale = static_cast<const float*>(adjoint ? p.d_sqrtW : p.d_rsqrtW);
  ModesTcArgs a;
  a.nb = p.nb;
  a.nmodes = nmodes;
  a.np = modes_np(p);
  a.nn = modes_nn(nmodes);
  a.nf = p.nf;
  a.mcount = mcount;
  a.m0 = m0;
  a.M = out_ld ? out_ld : (p.phi_ld && !adjoint) ? p.phi_ld : p.M;
  a.phioff = out_ld ? out_off : adjoint ? 0 : p.phi_off;
  a.ntp = (mcount + 127) / 128;
  a.qtile0 = qoff / 128;
  a.nitems = a.ntp * (f1 - f0);
  a.f0 = f0;
  a.box_bytes = (uint32_t)a.np * 128u;
  a.img_bytes = modes_img_bytes(a.np, a.nn);
  const int sms = p.num_sms > 0 ? p.num_sms : 148;
  int64_t grid = sms;
  if (p.modes_ctas > 0) grid = (int64_t)p.modes_ctas;   // tuning override: total CTAs
  grid = std::max<int64_t>(1, std::min<int64_t>(grid, a.nitems));
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p.device);
  a.nst = kMaxStages;
  while (a.nst > 2 && modes_tc_smem_stages(p, a.nst) > (size_t)optin) --a.nst;
  const size_t smem = modes_tc_smem_stages(p, a.nst);
  if (p.desc.precision == SPOD_PREC_BF16X3) {
    cudaError_t e = cudaFuncSetAttribute(k_modes_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_modes_tc<true><<<(unsigned)grid, kThreadsModes, smem, s>>>(p.tmap_hi2, p.tmap_lo2, a,
                                                                 static_cast<const uint8_t*>(p.d_bimg), scale,
                                                                 static_cast<float2*>(d_Phi), p.d_flags);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_modes_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_modes_tc<false><<<(unsigned)grid, kThreadsModes, smem, s>>>(p.tmap_hi2, p.tmap_hi2, a,
                                                                  static_cast<const uint8_t*>(p.d_bimg), scale,
                                                                  static_cast<float2*>(d_Phi), p.d_flags);
  }
  return cudaGetLastError();
}

}  // namespace spod
