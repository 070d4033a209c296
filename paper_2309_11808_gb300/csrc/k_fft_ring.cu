// Persistent block DFT (Eqs. blocks, blocks-ft, blocks-k) with a TMA ring, for
// nfft values without a compiled radix sequence (those use k_fft_pipe.cu).
//
// Persistent CTAs of 512 threads walk tiles of 16 spatial points; for each tile
// a CTA transforms the Welch blocks l = 0 .. nb-1 in order.  The tile's time
// rows arrive by TMA into a ring of nfft + step rows: block 0 loads nfft rows,
// each later block only its step new rows (the overlap is already resident),
// and the next block's rows are requested while the current block is
// transformed, so every sample of X is read from HBM once.  Per block: mean
// subtraction (double-float pair), window c w_n, two real point series packed
// into one complex sequence, an in-place shared-memory Stockham FFT following
// the plan's runtime radix list (8/4/2/3/5), the two real spectra separated,
// sqrt(W) folded in, and the output planes staged in shared memory and
// written by TMA bulk tensor stores (planar FP32 rows, or the 64-point blocked
// BF16 layout of the tensor-core path).
//
// Requires M * sizeof(element) to be a multiple of 16 bytes (TMA row stride);
// other shapes use the per-block kernel of k_fft.cu.
#include <type_traits>

#include "fft_common.cuh"
#include "tc_common.cuh"

namespace spod {
namespace {

using namespace fft;

constexpr int RTP = 16;          // points per tile
constexpr int RC = RTP / 2;      // complex columns (point pairs)
constexpr int RTHREADS = 512;

struct RingArgs {
  int64_t M, m0, mcount, chunk, mpad, ntiles;
  int64_t xoff;                     // column of X's first TMA column (tiled data)
  int nfft, step, nb, nf, boxr, ring;
  int stg_off;                      // byte offset of the output staging (from the ring start)
  int fbox, nfbox;                  // frequency rows per TMA store box, boxes per plane
  int pst;                          // staging plane stride in elements (nfbox * fbox * 16, 128-byte padded)
  int subtract_mean;
  FftPlan fp;
};

struct RingHdr {
  uint64_t full;
  int abort;
};

// In-place Stockham pass over RC interleaved sequences: every thread loads the
// inputs of its (at most MAXB) butterflies, the block synchronises, then every
// thread writes its outputs.  MAXB = ceil(NMAX * RC / (RAD * RTHREADS)).
template <int RAD, int MAXB>
__device__ __forceinline__ void pass_inplace(float2* __restrict__ buf, const float2* __restrict__ tw, int n, int Ns,
                                             int log2Ns) {
  const int nbut = n / RAD;
  const int stride_tw = n / (Ns * RAD);
  constexpr int BSTEP = RTHREADS / RC;
  const int col = threadIdx.x % RC;
  const int b0 = threadIdx.x / RC;
  float2 v[MAXB][RAD];
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    const int b = b0 + i * BSTEP;
    if (b < nbut) {
#pragma unroll
      for (int r = 0; r < RAD; ++r) v[i][r] = buf[(b + r * nbut) * RC + col];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    const int b = b0 + i * BSTEP;
    if (b < nbut) {
      int k, g;
      if (log2Ns >= 0) { k = b & (Ns - 1); g = b >> log2Ns; }
      else { g = b / Ns; k = b - g * Ns; }
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < RAD; ++r) v[i][r] = cmul(v[i][r], tw[r * k * stride_tw]);
      }
      dft_small<RAD, float2, float>(v[i]);
      const int base = g * Ns * RAD + k;
#pragma unroll
      for (int r = 0; r < RAD; ++r) buf[(base + r * Ns) * RC + col] = v[i][r];
    }
  }
  __syncthreads();
}

template <int NMAX, int RAD>
struct MaxB {
  static constexpr int value = (NMAX * RC + RAD * RTHREADS - 1) / (RAD * RTHREADS);
};


template <typename Tin, int OUTK, int NMAX>
__global__ void __launch_bounds__(RTHREADS, 1) k_fft_ring(const __grid_constant__ CUtensorMap xmap,
                                                          const __grid_constant__ CUtensorMap smap_hi,
                                                          const __grid_constant__ CUtensorMap smap_lo,
                                                          const float* __restrict__ win,
                                                          const float2* __restrict__ tw_g,
                                                          const float* __restrict__ sqrtW,
                                                          const double* __restrict__ mu, void* __restrict__ qout,
                                                          void* __restrict__ qout_lo, RingArgs a,
                                                          unsigned* __restrict__ gflags) {
  using namespace tc;
  extern __shared__ unsigned char smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  RingHdr* hdr = reinterpret_cast<RingHdr*>(sm);
  Tin* ring = reinterpret_cast<Tin*>(sm + 1024);                        // [ring rows][RTP]
  float2* buf = reinterpret_cast<float2*>(sm + 1024 + (size_t)a.ring * RTP * sizeof(Tin));
  float2* tw = buf + (size_t)a.nfft * RC;
  float* wsm = reinterpret_cast<float*>(tw + a.nfft);                   // c w_n
  float* swt = wsm + a.nfft;                                            // sqrt(W) of the tile
  // output staging, two buffers: [plane][nf][RTP] (planes: re, im [, re lo, im lo])
  constexpr int NPL = (OUTK == OUT_BF16X3) ? 4 : 2;
  using Tout = typename std::conditional<OUTK == OUT_NATIVE, float, __nv_bfloat16>::type;
  Tout* stg0 = reinterpret_cast<Tout*>(sm + 1024 + a.stg_off);
  const int stg_elems = NPL * a.pst;
  const int N = a.nfft, S = a.step;
  const int tid = threadIdx.x;
  const uint32_t bar = smem_u32(&hdr->full);
  volatile int* abort_flag = &hdr->abort;

  if (tid == 0) {
    mbar_init(bar, 1);
    hdr->abort = 0;
    fence_mbar_init();
  }
  for (int i = tid; i < N; i += RTHREADS) {
    tw[i] = tw_g[i];
    wsm[i] = win[i];
  }
  __syncthreads();

  const int64_t t_first = blockIdx.x;
  const int64_t t_step = gridDim.x;
  if (t_first >= a.ntiles) return;
  const uint32_t row_bytes = RTP * sizeof(Tin);

  // issue the TMA boxes for time rows [r0, r0 + nrows) of tile t into the ring
  auto issue = [&](int64_t t, int r0, int nrows) {
    mbar_arrive_expect_tx(bar, (uint32_t)nrows * row_bytes);
    const int x = (int)(a.m0 - a.xoff + t * RTP);
    for (int r = r0; r < r0 + nrows; r += a.boxr) {
      const int slot = r % a.ring;
      tma_load_2d(smem_u32(ring + (size_t)slot * RTP), &xmap, x, r, bar);
    }
  };
  if (tid == 0) {
    prefetch_tmap(&xmap);
    issue(t_first, 0, N);
  }

  const int j = tid % RC;            // copy phase: this thread's column (point pair)
  const int n0 = tid / RC;
  uint32_t phase = 0;
  bool last_ok = true;               // thread 0: its last wait saw the copy land
  uint32_t blk = 0;                  // blocks transformed by this CTA (staging buffer parity)
  for (int64_t t = t_first; t < a.ntiles; t += t_step) {
    const int64_t lm0 = t * RTP;
    const int64_t gm0 = a.m0 + lm0;
    float mhi0 = 0.f, mlo0 = 0.f, mhi1 = 0.f, mlo1 = 0.f;
    {
      const int64_t m = gm0 + 2 * j;
      const int64_t mend = a.m0 + a.mcount;
      if (a.subtract_mean && m < mend) { const double d = mu[m]; mhi0 = (float)d; mlo0 = (float)(d - (double)mhi0); }
      if (a.subtract_mean && m + 1 < mend) {
        const double d = mu[m + 1]; mhi1 = (float)d; mlo1 = (float)(d - (double)mhi1);
      }
      if (tid < RTP) swt[tid] = (lm0 + tid < a.mcount) ? sqrtW[gm0 + tid] : 0.f;
    }
    for (int l = 0; l < a.nb; ++l) {
      last_ok = mbar_wait(bar, phase & 1, abort_flag, gflags);
      ++phase;
      __syncthreads();
      if (hdr->abort) break;
      // ---- ring rows -> FFT buffer (mean, window, pack two points)
      const int rbase = l * S;
      const int rb = rbase % a.ring;
      for (int n = n0; n < N; n += RTHREADS / RC) {
        int slot = rb + n;
        if (slot >= a.ring) slot -= a.ring;
        const Tin* rp = ring + slot * RTP + 2 * j;
        const float x0 = (to_f32<Tin>(rp[0]) - mhi0) - mlo0;
        const float x1 = (to_f32<Tin>(rp[1]) - mhi1) - mlo1;
        const float wn = wsm[n];
        buf[n * RC + j] = make_float2(x0 * wn, x1 * wn);
      }
      __syncthreads();
      // ---- request the next rows (ring slots of rows no longer needed)
      if (tid == 0) {
        if (l + 1 < a.nb) {
          issue(t, rbase + N, S);
        } else if (t + t_step < a.ntiles) {
          issue(t + t_step, 0, N);
        }
      }
      // ---- FFT (in place)
      {
        int Ns = 1, log2Ns = 0;
        for (int ps = 0; ps < a.fp.npass; ++ps) {
          const int rad = a.fp.radix[ps];
          switch (rad) {
            case 8: pass_inplace<8, MaxB<NMAX, 8>::value>(buf, tw, N, Ns, log2Ns); break;
            case 4: pass_inplace<4, MaxB<NMAX, 4>::value>(buf, tw, N, Ns, log2Ns); break;
            case 2: pass_inplace<2, MaxB<NMAX, 2>::value>(buf, tw, N, Ns, log2Ns); break;
            case 3: pass_inplace<3, MaxB<NMAX, 3>::value>(buf, tw, N, Ns, log2Ns); break;
            default: pass_inplace<5, MaxB<NMAX, 5>::value>(buf, tw, N, Ns, log2Ns); break;
          }
          Ns *= rad;
          if (log2Ns >= 0) log2Ns = (rad == 2) ? log2Ns + 1 : (rad == 4) ? log2Ns + 2 : (rad == 8) ? log2Ns + 3 : -1;
        }
      }
      const float2* src = buf;
      // ---- separate the two real spectra of each column, fold sqrt(W), stage the
      // output planes [plane][f][16 points] in shared memory, store them by TMA
      Tout* stg = stg0 + (size_t)(blk & 1) * stg_elems;
      if (tid == 0) tma_store_wait_read<1>();      // the stores that last read this buffer are done
      __syncthreads();
      const int pp = tid % RC;
      const int f0 = tid / RC;
      constexpr int FSTEP = RTHREADS / RC;
      const float sa = swt[2 * pp], sb = swt[2 * pp + 1];
      for (int f = f0; f < a.nf; f += FSTEP) {
        const float2 zf = src[f * RC + pp];
        const float2 zc = src[((f == 0) ? 0 : N - f) * RC + pp];
        // even point: (Z[f] + conj Z[N-f]) / 2 ; odd point: (Z[f] - conj Z[N-f]) / (2i)
        const float ra = 0.5f * (zf.x + zc.x) * sa, ia = 0.5f * (zf.y - zc.y) * sa;
        const float rb = 0.5f * (zf.y + zc.y) * sb, ib = -0.5f * (zf.x - zc.x) * sb;
        const int e = f * RTP + 2 * pp;
        if constexpr (OUTK == OUT_NATIVE) {
          *reinterpret_cast<float2*>(stg + e) = make_float2(ra, rb);
          *reinterpret_cast<float2*>(stg + a.pst + e) = make_float2(ia, ib);
        } else {
          const __nv_bfloat162 hr = __floats2bfloat162_rn(ra, rb);
          const __nv_bfloat162 hi = __floats2bfloat162_rn(ia, ib);
          *reinterpret_cast<__nv_bfloat162*>(stg + e) = hr;
          *reinterpret_cast<__nv_bfloat162*>(stg + a.pst + e) = hi;
          if constexpr (OUTK == OUT_BF16X3) {
            const float2 fr = __bfloat1622float2(hr), fi = __bfloat1622float2(hi);
            *reinterpret_cast<__nv_bfloat162*>(stg + 2 * a.pst + e) = __floats2bfloat162_rn(ra - fr.x, rb - fr.y);
            *reinterpret_cast<__nv_bfloat162*>(stg + 3 * a.pst + e) = __floats2bfloat162_rn(ia - fi.x, ib - fi.y);
          }
        }
      }
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) {
        // rows: re = l, im = nb + l of every frequency; boxes of fbox frequencies
        // (the staged planes cover nfbox * fbox rows, so every box read stays inside them;
        // frequencies past nf are clipped by the store)
        for (int pl = 0; pl < NPL; ++pl) {
          const CUtensorMap* mp = (pl < 2) ? &smap_hi : &smap_lo;
          const int row = (pl & 1) ? a.nb + l : l;
          for (int b = 0; b < a.nfbox; ++b) {
            const uint32_t src = smem_u32(stg + (size_t)pl * a.pst + (size_t)b * a.fbox * RTP);
            if constexpr (OUTK == OUT_NATIVE) {
              tma_store_3d(mp, (int)lm0, row, b * a.fbox, src);
            } else {   // blocked BF16 layout: point within the 64-point block, block index last
              tma_store_4d(mp, (int)(lm0 % kQBlock), row, b * a.fbox, (int)(lm0 / kQBlock), src);
            }
          }
        }
        tma_store_commit();
      }
      ++blk;
      __syncthreads();
    }
    if (hdr->abort) break;
  }
  // a request issued before an abort must land before the CTA exits, and the
  // output stores must have finished reading shared memory
  if (tid == 0 && !last_ok) mbar_drain(bar, (phase - 1) & 1, gflags);
  if (tid == 0) tma_store_wait_all<0>();
}

template <typename Tin, int OUTK, int NMAX>
cudaError_t launch_ring_n(const spod_plan_s& p, const CUtensorMap& xmap, int64_t m0, int64_t mcount,
                          cudaStream_t s) {
  RingArgs a;
  a.M = p.M; a.m0 = m0; a.mcount = mcount; a.chunk = p.chunk_points;
  a.xoff = p.x_off;
  a.mpad = std::min<int64_t>(p.chunk_points, (mcount + 63) / 64 * 64);
  a.ntiles = a.mpad / RTP;
  a.nfft = p.nfft; a.step = p.step; a.nb = p.nb; a.nf = p.nf;
  a.boxr = p.ring_boxr;
  a.ring = p.nfft + p.step;
  a.subtract_mean = p.desc.subtract_mean;
  a.fp = p.fft;
  a.stg_off = (int)fft_ring_stage_offset(p);
  a.fbox = p.fst_fbox;
  a.nfbox = (p.nf + p.fst_fbox - 1) / p.fst_fbox;
  a.pst = (int)fft_ring_plane_elems(p);
  const size_t smem = fft_ring_smem_bytes(p);
  auto kern = k_fft_ring<Tin, OUTK, NMAX>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RTHREADS, smem);
  per_sm = std::max(1, per_sm);
  const int grid = (int)std::min<int64_t>(a.ntiles, (int64_t)(p.num_sms > 0 ? p.num_sms : 148) * per_sm);
  kern<<<grid, RTHREADS, smem, s>>>(xmap, p.tmap_fst_hi, p.tmap_fst_lo, static_cast<const float*>(p.d_win),
                                    static_cast<const float2*>(p.d_tw),
                                    static_cast<const float*>(p.d_sqrtW), p.d_mu, p.d_qhat, p.d_qlo, a, p.d_flags);
  return cudaGetLastError();
}

template <typename Tin, int OUTK>
cudaError_t launch_ring_t(const spod_plan_s& p, const CUtensorMap& xmap, int64_t m0, int64_t mcount,
                          cudaStream_t s) {
  if (p.nfft <= 512) return launch_ring_n<Tin, OUTK, 512>(p, xmap, m0, mcount, s);
  return launch_ring_n<Tin, OUTK, 1024>(p, xmap, m0, mcount, s);
}

template <typename Tin>
cudaError_t launch_ring_in(const spod_plan_s& p, const CUtensorMap& xmap, int64_t m0, int64_t mcount,
                           cudaStream_t s) {
  if (p.desc.precision == SPOD_PREC_BF16X3) return launch_ring_t<Tin, OUT_BF16X3>(p, xmap, m0, mcount, s);
  if (p.desc.precision == SPOD_PREC_BF16) return launch_ring_t<Tin, OUT_BF16>(p, xmap, m0, mcount, s);
  return launch_ring_t<Tin, OUT_NATIVE>(p, xmap, m0, mcount, s);
}

}  // namespace

// Byte offset (from the ring start) of the output staging area, 128-byte aligned.
size_t fft_ring_stage_offset(const spod_plan_s& p) {
  const size_t el = p.desc.in_dtype == SPOD_F64 ? 8 : (p.desc.in_dtype == SPOD_F32 ? 4 : 2);
  const size_t pre = (size_t)(p.nfft + p.step) * RTP * el + sizeof(float2) * ((size_t)p.nfft * RC + p.nfft) +
                     sizeof(float) * (p.nfft + RTP);
  return (pre + 127) & ~size_t(127);
}

// Staging plane stride (elements): whole store boxes of fst_fbox frequency rows x 16
// points, padded to 128 bytes.
size_t fft_ring_plane_elems(const spod_plan_s& p) {
  const size_t oel = p.tensor ? 2 : 4;
  const size_t nbox = (p.nf + p.fst_fbox - 1) / p.fst_fbox;
  const size_t bytes = nbox * p.fst_fbox * RTP * oel;
  return ((bytes + 127) & ~size_t(127)) / oel;
}

size_t fft_ring_smem_bytes(const spod_plan_s& p) {
  const size_t npl = p.desc.precision == SPOD_PREC_BF16X3 ? 4 : 2;
  const size_t oel = p.tensor ? 2 : 4;
  return 1024 + 1024 + fft_ring_stage_offset(p) + 2 * npl * fft_ring_plane_elems(p) * oel;
}

bool fft_ring_usable(const spod_plan_s& p, int smem_optin) {
  if (p.f64) return false;
  const size_t el = p.desc.in_dtype == SPOD_F64 ? 8 : (p.desc.in_dtype == SPOD_F32 ? 4 : 2);
  if ((p.M * (int64_t)el) % 16 != 0) return false;        // TMA row stride
  if (p.ring_boxr <= 0 || p.nfft > 1024 || !p.fst_maps) return false;
  return fft_ring_smem_bytes(p) <= (size_t)smem_optin;
}

cudaError_t launch_fft_ring_chunk(const spod_plan_s& p, const CUtensorMap& xmap, int64_t m0, int64_t mcount,
                                  cudaStream_t s) {
  if (p.desc.in_dtype == SPOD_F64) return launch_ring_in<double>(p, xmap, m0, mcount, s);
  if (p.desc.in_dtype == SPOD_F32) return launch_ring_in<float>(p, xmap, m0, mcount, s);
  return launch_ring_in<__nv_bfloat16>(p, xmap, m0, mcount, s);
}

}  // namespace spod
