// Persistent block DFT (Eqs. blocks, blocks-ft, blocks-k) for the nfft values
// with a compiled radix sequence (256, 384, 512, 720).
//
// Complex data (CPLX) runs through the same ring and passes as an array of
// 2M interleaved real components: a column of the transform then holds one
// complex point (its real and imaginary parts) instead of two real points,
// and the output phase keeps all nfft bins with no separation.
//
// Persistent CTAs walk tiles of TP spatial points (TP = 32: one 512-thread CTA
// per SM; TP = 16: two 256-thread CTAs per SM, for nfft = 720 and FP64 input,
// whose rings do not fit twice); each CTA transforms the Welch blocks
// l = 0 .. nb-1 of its tile in order.  The wider tile halves the number of
// 128-byte lines per stored byte in the output phase (a line of the BF16
// blocked layout holds 64 points of one row) and makes every TMA ring row a
// full 128-byte line.  The tile's
// time rows arrive by TMA into a ring of exactly nfft rows: block 0 loads
// nfft rows, each later block only its step new rows, written over the rows
// the previous block no longer needs, so every sample of X is read from HBM
// once and the request for block l+1 is in flight while block l is
// transformed.
//
// Per block the Stockham passes run out of place between two shared-memory
// buffers, so a pass needs one barrier (after its stores) instead of two:
//   pass 0   reads the ring directly and applies the mean (double-float pair)
//            and the window c w_n while loading its butterfly inputs;
//   pass i   buffer -> other buffer, twiddled radix-R butterflies;
//   output   the two real spectra packed in each complex column are
//            separated, sqrt(W) is folded in, and the planar rows
//            Q[f][l][m] (re) and Q[f][nb+l][m] (im) are stored directly.
// The buffer roles alternate between blocks when the pass count is odd, so
// the next block's pass 0 never writes the buffer the output phase reads and
// no barrier is needed between them.
#include <type_traits>

#include "fft_common.cuh"
#include "tc_common.cuh"

namespace spod {
namespace {

using namespace fft;

// Tile geometry: TP points, TP/2 complex columns, 16 threads per point.
template <int TP>
struct Geo {
  static constexpr int PTP = TP;                   // points per tile
  static constexpr int PC = TP / 2;                // complex columns (point pairs)
  static constexpr int THREADS = 16 * TP;
  static constexpr int BSTEP = THREADS / PC;       // butterflies between a thread's consecutive ones (32)
  static constexpr int OUTCP = PC / 2;             // column pairs per tile
  static constexpr int OUTFSTEP = THREADS / OUTCP; // bins between a thread's consecutive ones (64)
};

struct PipeArgs {
  int64_t m0, mcount, chunk, ntiles;
  int64_t xoff;                      // column of X's first TMA column (tiled data)
  int step, nb, nf, boxr;
  int subtract_mean;
  int qrows;                         // Qhat rows per frequency (blocked layout)
  // time mean folded into the transform (real data): a provisional centre
  // c (the mean of kCentreSamples evenly spaced snapshots of the column) is
  // subtracted instead of the mean, the sum of x - c over all nt snapshots
  // accumulated, mu = c + mean(x - c) written to mu_out and
  // rho = sqrt(W) mean(x - c) to Qhat row 2 nb of every frequency
  int fold;
  int64_t nt, tail0;                 // snapshots; first snapshot in no block
  const void* xg;                    // X itself (tail samples), row stride xld, column of point lm: xc0 + lm
  int64_t xld, xc0;
  double* mu_out;
};

// Snapshots that give the provisional centre of a column when the mean is
// folded: the closer c is to mu, the smaller the rank-one correction and the
// cancellation it brings to the low bins (the centre's offset from mu enters
// the uncorrected spectra times sum_n w_n)
constexpr int kCentreSamples = 128;

// Compensated (Kahan) FP32 sum: s + (-c) carries the running total to about
// one rounding of the result.  The folded mean's sums use it instead of FP64
// adds, which run at a small fraction of the FP32 rate on this part.
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

struct PipeHdr {
  uint64_t full;
  int abort;
};

template <typename Tin> struct PairLoad;
template <> struct PairLoad<float> {
  static __device__ __forceinline__ float2 get(const float* p) { return *reinterpret_cast<const float2*>(p); }
};
template <> struct PairLoad<__nv_bfloat16> {
  static __device__ __forceinline__ float2 get(const __nv_bfloat16* p) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
  }
};
template <> struct PairLoad<double> {
  static __device__ __forceinline__ float2 get(const double* p) {
    const double2 d = *reinterpret_cast<const double2*>(p);
    return make_float2((float)d.x, (float)d.y);
  }
};

// Pass 0 (Ns = 1, no twiddles): butterfly inputs come from the ring rows of
// the current block with the mean removed and the window applied.  Element r
// of butterfly b is sample n = b + r N / RAD; with FOLD the elements with
// r >= rthr (a block-uniform bound) are also summed into acc0 / acc1.
template <typename Tin, int TP, int N, int RAD, bool FOLD>
__device__ __forceinline__ void pass_first(const Tin* __restrict__ ring, int rb, float2* __restrict__ dst,
                                           const float* __restrict__ wsm, float mhi0, float mlo0, float mhi1,
                                           float mlo1, int rthr, float& acc0, float& acc1) {
  constexpr int PTP = Geo<TP>::PTP, PC = Geo<TP>::PC, PBSTEP = Geo<TP>::BSTEP;
  constexpr int nbut = N / RAD;
  constexpr int MAXB = (nbut + PBSTEP - 1) / PBSTEP;
  const int col = threadIdx.x % PC;
  const int b0 = threadIdx.x / PC;
  float2 v[MAXB][RAD];
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    const int b = b0 + i * PBSTEP;
    if (nbut % PBSTEP == 0 || b < nbut) {
#pragma unroll
      for (int r = 0; r < RAD; ++r) {
        const int n = b + r * nbut;
        int slot = rb + n;
        if (slot >= N) slot -= N;
        const float2 x = PairLoad<Tin>::get(ring + slot * PTP + 2 * col);
        const float wn = wsm[n];
        const float d0 = (x.x - mhi0) - mlo0, d1 = (x.y - mhi1) - mlo1;
        if (FOLD && r >= rthr) {           // a snapshot no earlier block held
          acc0 += d0;
          acc1 += d1;
        }
        v[i][r] = make_float2(d0 * wn, d1 * wn);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    const int b = b0 + i * PBSTEP;
    if (nbut % PBSTEP == 0 || b < nbut) {
      dft_small<RAD, float2, float>(v[i]);
#pragma unroll
      for (int r = 0; r < RAD; ++r) dst[(b * RAD + r) * PC + col] = v[i][r];
    }
  }
}

// Out-of-place Stockham pass with compile-time radix and stride.
template <int TP, int N, int RAD, int NS>
__device__ __forceinline__ void pass_oop(const float2* __restrict__ src, float2* __restrict__ dst,
                                         const float2* __restrict__ tw) {
  constexpr int PC = Geo<TP>::PC, PBSTEP = Geo<TP>::BSTEP;
  constexpr int nbut = N / RAD;
  constexpr int MAXB = (nbut + PBSTEP - 1) / PBSTEP;
  constexpr int stw = N / (NS * RAD);
  const int col = threadIdx.x % PC;
  const int b0 = threadIdx.x / PC;
  float2 v[MAXB][RAD];
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    const int b = b0 + i * PBSTEP;
    if (nbut % PBSTEP == 0 || b < nbut) {
#pragma unroll
      for (int r = 0; r < RAD; ++r) v[i][r] = src[(b + r * nbut) * PC + col];
    }
  }
  // when PBSTEP is a multiple of NS all of this thread's butterflies share k
  float2 tk[RAD];
  if constexpr (PBSTEP % NS == 0) {
    const int k = b0 % NS;
#pragma unroll
    for (int r = 1; r < RAD; ++r) tk[r] = tw[r * k * stw];
  }
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    const int b = b0 + i * PBSTEP;
    if (nbut % PBSTEP == 0 || b < nbut) {
      const int k = b % NS, g = b / NS;
#pragma unroll
      for (int r = 1; r < RAD; ++r) v[i][r] = cmul(v[i][r], (PBSTEP % NS == 0) ? tk[r] : tw[r * k * stw]);
      dft_small<RAD, float2, float>(v[i]);
      const int base = g * NS * RAD + k;
#pragma unroll
      for (int r = 0; r < RAD; ++r) dst[(base + r * NS) * PC + col] = v[i][r];
    }
  }
}

// Passes 1 .. P-1, each followed by a barrier; returns the buffer holding
// the spectrum.
template <int TP, int N, int NS, int R0, int... RS>
__device__ __forceinline__ const float2* run_rest(float2* src, float2* dst, const float2* tw) {
  pass_oop<TP, N, R0, NS>(src, dst, tw);
  __syncthreads();
  if constexpr (sizeof...(RS) > 0) {
    return run_rest<TP, N, NS * R0, RS...>(dst, src, tw);
  } else {
    return dst;
  }
}

// Radix sequences (first radix, then the rest).
template <int N> struct PSeq;
template <> struct PSeq<256> {
  static constexpr int R0 = 8, P = 3;
  template <int TP>
  static __device__ __forceinline__ const float2* rest(float2* a, float2* b, const float2* t) {
    return run_rest<TP, 256, 8, 8, 4>(a, b, t);
  }
};
template <> struct PSeq<384> {
  static constexpr int R0 = 8, P = 4;
  template <int TP>
  static __device__ __forceinline__ const float2* rest(float2* a, float2* b, const float2* t) {
    return run_rest<TP, 384, 8, 8, 2, 3>(a, b, t);
  }
};
template <> struct PSeq<512> {
  static constexpr int R0 = 8, P = 3;
  template <int TP>
  static __device__ __forceinline__ const float2* rest(float2* a, float2* b, const float2* t) {
    return run_rest<TP, 512, 8, 8, 8>(a, b, t);
  }
};
template <> struct PSeq<720> {
  static constexpr int R0 = 8, P = 5;
  template <int TP>
  static __device__ __forceinline__ const float2* rest(float2* a, float2* b, const float2* t) {
    return run_rest<TP, 720, 8, 2, 3, 3, 5>(a, b, t);
  }
};

// Separate the two real spectra of each column (even point: (Z[f] + conj
// Z[N-f]) / 2, odd point: (Z[f] - conj Z[N-f]) / 2i), fold sqrt(W) (sw carries
// the 1/2) and store rows re = l and im = nb + l of every frequency.  A thread
// takes two adjacent columns (four points): 16-byte shared loads, and one
// 16-byte (FP32) or 8-byte (BF16) store per output plane and frequency.
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ float bf16_lo_f(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi_f(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// Complex data: column c is point c of the tile (lp0 = its first point);
// a thread takes two adjacent columns of bins f0, f0 + 64, ... over all N
// bins and stores them with sqrt(W) (sw, no 1/2) as two-point rows.
template <int OUTK, int TP, int N>
__device__ __forceinline__ void output_phase_cplx(const float2* __restrict__ src, const PipeArgs& a, int l,
                                                  int64_t lp0, const float (&sw)[4], void* __restrict__ qout,
                                                  void* __restrict__ qlo) {
  constexpr int kOutCp = Geo<TP>::OUTCP, kOutFStep = Geo<TP>::OUTFSTEP;
  const int cp = threadIdx.x % kOutCp;
  const int f0 = threadIdx.x / kOutCp;
  constexpr bool BLK = OUTK != OUT_NATIVE;
  const int64_t rs = BLK ? (int64_t)kQBlock : a.chunk;
  const int64_t rowstride = (int64_t)(BLK ? a.qrows : 2 * a.nb) * rs;
  const int64_t imoff = (int64_t)a.nb * rs;
  int64_t o = BLK ? qhat_blocked_offset(a.nf, a.qrows, f0, l, lp0 + 2 * cp)
                  : ((int64_t)f0 * 2 * a.nb + l) * a.chunk + lp0 + 2 * cp;
  const float4* src4 = reinterpret_cast<const float4*>(src);
  constexpr int kIters = (N + kOutFStep - 1) / kOutFStep;
#pragma unroll
  for (int it = 0; it < kIters; ++it) {
    const int f = f0 + it * kOutFStep;
    if (f >= N) break;
    if (it > 0) o += kOutFStep * rowstride;
    const float4 z = src4[f * kOutCp + cp];                       // points 2cp, 2cp+1 at bin f
    const float r0 = z.x * sw[0], i0 = z.y * sw[0];
    const float r1 = z.z * sw[1], i1 = z.w * sw[1];
    if constexpr (OUTK == OUT_NATIVE) {
      float* q = static_cast<float*>(qout);
      *reinterpret_cast<float2*>(q + o) = make_float2(r0, r1);
      *reinterpret_cast<float2*>(q + o + imoff) = make_float2(i0, i1);
    } else {
      __nv_bfloat16* qh = static_cast<__nv_bfloat16*>(qout);
      const uint32_t hr = pack_bf16x2(r0, r1), hi = pack_bf16x2(i0, i1);
      *reinterpret_cast<uint32_t*>(qh + o) = hr;
      *reinterpret_cast<uint32_t*>(qh + o + imoff) = hi;
      if constexpr (OUTK == OUT_BF16X3) {
        __nv_bfloat16* ql = static_cast<__nv_bfloat16*>(qlo);
        *reinterpret_cast<uint32_t*>(ql + o) = pack_bf16x2(r0 - bf16_lo_f(hr), r1 - bf16_hi_f(hr));
        *reinterpret_cast<uint32_t*>(ql + o + imoff) = pack_bf16x2(i0 - bf16_lo_f(hi), i1 - bf16_hi_f(hi));
      }
    }
  }
}

template <int OUTK, int TP, int N>
__device__ __forceinline__ void output_phase(const float2* __restrict__ src, const PipeArgs& a, int l,
                                             int64_t lm0, const float (&sw)[4], void* __restrict__ qout,
                                             void* __restrict__ qlo) {
  constexpr int kOutCp = Geo<TP>::OUTCP, kOutFStep = Geo<TP>::OUTFSTEP;
  const int cp = threadIdx.x % kOutCp;
  const int f0 = threadIdx.x / kOutCp;
  // FP32 planes are planar [nf][2 nb][chunk]; BF16 planes are blocked by 64
  // points, [chunk / 64][nf][2 nb][64] (see qhat_blocked_offset)
  constexpr bool BLK = OUTK != OUT_NATIVE;
  const int64_t rs = BLK ? (int64_t)kQBlock : a.chunk;           // row stride
  const int64_t rowstride = (int64_t)(BLK ? a.qrows : 2 * a.nb) * rs;   // one frequency
  const int64_t imoff = (int64_t)a.nb * rs;
  int64_t o = BLK ? qhat_blocked_offset(a.nf, a.qrows, f0, l, lm0 + 4 * cp)
                  : ((int64_t)f0 * 2 * a.nb + l) * a.chunk + lm0 + 4 * cp;
  const float4* src4 = reinterpret_cast<const float4*>(src);
  // compile-time trip count (nf = N/2 + 1): the iterations' loads overlap
  constexpr int kIters = (N / 2 + 1 + kOutFStep - 1) / kOutFStep;
#pragma unroll
  for (int it = 0; it < kIters; ++it) {
    const int f = f0 + it * kOutFStep;
    if (f >= a.nf) break;
    if (it > 0) o += kOutFStep * rowstride;
    const float4 zf = src4[f * kOutCp + cp];                        // columns 2cp, 2cp+1 at bin f
    const float4 zc = src4[((f == 0) ? 0 : N - f) * kOutCp + cp];   // ... at bin N-f
    // points 4cp, 4cp+1 (column 2cp) and 4cp+2, 4cp+3 (column 2cp+1)
    const float r0 = (zf.x + zc.x) * sw[0], i0 = (zf.y - zc.y) * sw[0];
    const float r1 = (zf.y + zc.y) * sw[1], i1 = (zc.x - zf.x) * sw[1];
    const float r2 = (zf.z + zc.z) * sw[2], i2 = (zf.w - zc.w) * sw[2];
    const float r3 = (zf.w + zc.w) * sw[3], i3 = (zc.z - zf.z) * sw[3];
    if constexpr (OUTK == OUT_NATIVE) {
      float* q = static_cast<float*>(qout);
      *reinterpret_cast<float4*>(q + o) = make_float4(r0, r1, r2, r3);
      *reinterpret_cast<float4*>(q + o + imoff) = make_float4(i0, i1, i2, i3);
    } else {
      __nv_bfloat16* qh = static_cast<__nv_bfloat16*>(qout);
      const uint32_t hr01 = pack_bf16x2(r0, r1), hr23 = pack_bf16x2(r2, r3);
      const uint32_t hi01 = pack_bf16x2(i0, i1), hi23 = pack_bf16x2(i2, i3);
      *reinterpret_cast<uint2*>(qh + o) = make_uint2(hr01, hr23);
      *reinterpret_cast<uint2*>(qh + o + imoff) = make_uint2(hi01, hi23);
      if constexpr (OUTK == OUT_BF16X3) {
        __nv_bfloat16* ql = static_cast<__nv_bfloat16*>(qlo);
        const uint32_t lr01 = pack_bf16x2(r0 - bf16_lo_f(hr01), r1 - bf16_hi_f(hr01));
        const uint32_t lr23 = pack_bf16x2(r2 - bf16_lo_f(hr23), r3 - bf16_hi_f(hr23));
        const uint32_t li01 = pack_bf16x2(i0 - bf16_lo_f(hi01), i1 - bf16_hi_f(hi01));
        const uint32_t li23 = pack_bf16x2(i2 - bf16_lo_f(hi23), i3 - bf16_hi_f(hi23));
        *reinterpret_cast<uint2*>(ql + o) = make_uint2(lr01, lr23);
        *reinterpret_cast<uint2*>(ql + o + imoff) = make_uint2(li01, li23);
      }
    }
  }
}

// ---------------------------------------------------------------- nfft = 512 in two passes
// n = 32 n1 + n2, k = k1 + 16 k2:
//   X[k1 + 16 k2] = sum_n2 W32^(n2 k2) W512^(n2 k1) sum_n1 x[32 n1 + n2] W16^(n1 k1).
// Pass A: thread (column, n2) takes its 16 samples from the ring, a 16-point
// DFT in registers, the twiddle W512^(n2 k1), and stores Y[k1][n2].  Pass B:
// thread (column, k1, h) takes Y[k1][2m + h], m < 16, and a 16-point DFT
// gives U_h[k1][k2] (k2 < 16); the remaining radix-2 step,
//   X[k1 + 16 k2] = U_0 + W32^k2 U_1,  X[k1 + 16 (k2 + 16)] = U_0 - W32^k2 U_1,
// is taken by the output phase, which needs X[f], X[N - f], X[256 - f] and
// X[256 + f] together anyway to separate the two real series of a column.
// Per element: one ring read, two shared-memory writes and two reads (the
// three-pass form: three writes and three reads), two barriers per block.

// 16-point forward DFT in registers (radix 4 x 4).
__device__ __forceinline__ void dft16(float2* v) {
  constexpr float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, r2 = 0.70710678118654752440f;
  float2 a[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float2 t[4] = {v[q], v[q + 4], v[q + 8], v[q + 12]};
    dft_small<4, float2, float>(t);
#pragma unroll
    for (int r = 0; r < 4; ++r) a[q][r] = t[r];
  }
  // a[q][r] *= W16^(q r)
  const float2 w1 = make_float2(c1, -s1), w3 = make_float2(s1, -c1), w9 = make_float2(-c1, s1);
  a[1][1] = cmul(a[1][1], w1);
  a[1][2] = make_float2(r2 * (a[1][2].x + a[1][2].y), r2 * (a[1][2].y - a[1][2].x));   // W^2
  a[1][3] = cmul(a[1][3], w3);
  a[2][1] = make_float2(r2 * (a[2][1].x + a[2][1].y), r2 * (a[2][1].y - a[2][1].x));   // W^2
  a[2][2] = mul_mi(a[2][2]);                                                            // W^4
  a[2][3] = make_float2(r2 * (a[2][3].y - a[2][3].x), -r2 * (a[2][3].x + a[2][3].y));  // W^6
  a[3][1] = cmul(a[3][1], w3);
  a[3][2] = make_float2(r2 * (a[3][2].y - a[3][2].x), -r2 * (a[3][2].x + a[3][2].y));  // W^6
  a[3][3] = cmul(a[3][3], w9);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    float2 t[4] = {a[0][r], a[1][r], a[2][r], a[3][r]};
    dft_small<4, float2, float>(t);
#pragma unroll
    for (int q = 0; q < 4; ++q) v[r + 4 * q] = t[q];
  }
}

// Pass A (see above).  With FOLD the samples n1 >= n1thr (a block-uniform
// bound) are also summed into acc0 / acc1.
template <typename Tin, int TP, bool FOLD>
__device__ __forceinline__ void pass_a512(const Tin* __restrict__ ring, int rb, float2* __restrict__ dst,
                                          const float* __restrict__ wsm, const float2* __restrict__ tw, float mhi0,
                                          float mlo0, float mhi1, float mlo1, int n1thr, float& acc0,
                                          float& acc1) {
  constexpr int N = 512, PTP = Geo<TP>::PTP, PC = Geo<TP>::PC;
  const int col = threadIdx.x % PC;
  const int n2 = threadIdx.x / PC;
  float2 v[16];
  const int s0 = rb + n2;
#pragma unroll
  for (int n1 = 0; n1 < 16; ++n1) {
    const int n = 32 * n1 + n2;
    const int slot = (s0 + 32 * n1) & (N - 1);
    const float2 x = PairLoad<Tin>::get(ring + slot * PTP + 2 * col);
    const float wn = wsm[n];
    const float d0 = (x.x - mhi0) - mlo0, d1 = (x.y - mhi1) - mlo1;
    if (FOLD && n1 >= n1thr) {
      acc0 += d0;
      acc1 += d1;
    }
    v[n1] = make_float2(d0 * wn, d1 * wn);
  }
  dft16(v);
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], tw[n2 * k1]);
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) dst[(k1 * 32 + n2) * PC + col] = v[k1];
}

// Pass B (see above): U_h[k1][k2] at row (h * 16 + k1) * 16 + k2.
template <int TP>
__device__ __forceinline__ void pass_b512(const float2* __restrict__ src, float2* __restrict__ dst) {
  constexpr int PC = Geo<TP>::PC;
  const int col = threadIdx.x % PC;
  const int j = threadIdx.x / PC;
  const int k1 = j >> 1, h = j & 1;
  float2 v[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) v[m] = src[(k1 * 32 + 2 * m + h) * PC + col];
  dft16(v);
  const int base = (h * 16 + k1) * 16;
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) dst[(base + k2) * PC + col] = v[k2];
}

// Store the one-sided spectra of the four points of column pair cp at bin f
// from z = X[f] and zc = X[N - f] of its two complex columns (float4 = two
// columns): the even point of a column is (z + conj zc) / 2, the odd one
// (z - conj zc) / 2i; sw carries sqrt(W) / 2.
template <int OUTK>
__device__ __forceinline__ void store_bin4(const float4 z, const float4 zc, const float (&sw)[4], const PipeArgs& a,
                                           int64_t o, void* __restrict__ qout, void* __restrict__ qlo) {
  const float r0 = (z.x + zc.x) * sw[0], i0 = (z.y - zc.y) * sw[0];
  const float r1 = (z.y + zc.y) * sw[1], i1 = (zc.x - z.x) * sw[1];
  const float r2 = (z.z + zc.z) * sw[2], i2 = (z.w - zc.w) * sw[2];
  const float r3 = (z.w + zc.w) * sw[3], i3 = (zc.z - z.z) * sw[3];
  if constexpr (OUTK == OUT_NATIVE) {
    float* q = static_cast<float*>(qout);
    *reinterpret_cast<float4*>(q + o) = make_float4(r0, r1, r2, r3);
    *reinterpret_cast<float4*>(q + o + (int64_t)a.nb * a.chunk) = make_float4(i0, i1, i2, i3);
  } else {
    const int64_t imoff = (int64_t)a.nb * kQBlock;
    __nv_bfloat16* qh = static_cast<__nv_bfloat16*>(qout);
    const uint32_t hr01 = pack_bf16x2(r0, r1), hr23 = pack_bf16x2(r2, r3);
    const uint32_t hi01 = pack_bf16x2(i0, i1), hi23 = pack_bf16x2(i2, i3);
    *reinterpret_cast<uint2*>(qh + o) = make_uint2(hr01, hr23);
    *reinterpret_cast<uint2*>(qh + o + imoff) = make_uint2(hi01, hi23);
    if constexpr (OUTK == OUT_BF16X3) {
      __nv_bfloat16* ql = static_cast<__nv_bfloat16*>(qlo);
      const uint32_t lr01 = pack_bf16x2(r0 - bf16_lo_f(hr01), r1 - bf16_hi_f(hr01));
      const uint32_t lr23 = pack_bf16x2(r2 - bf16_lo_f(hr23), r3 - bf16_hi_f(hr23));
      const uint32_t li01 = pack_bf16x2(i0 - bf16_lo_f(hi01), i1 - bf16_hi_f(hi01));
      const uint32_t li23 = pack_bf16x2(i2 - bf16_lo_f(hi23), i3 - bf16_hi_f(hi23));
      *reinterpret_cast<uint2*>(ql + o) = make_uint2(lr01, lr23);
      *reinterpret_cast<uint2*>(ql + o + imoff) = make_uint2(li01, li23);
    }
  }
}

__device__ __forceinline__ float4 c2add(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ float4 c2sub(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
// both complex columns of a float4 times w
__device__ __forceinline__ float4 c2mul(float4 a, float2 w) {
  return make_float4(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x, a.z * w.x - a.w * w.y, a.z * w.y + a.w * w.x);
}

// Output phase of the two-pass form: item j = f in [0, 128] of column pair cp
// gives bins f and 256 - f.  With (k1, k2) = (f mod 16, f / 16) and the
// partner (k1', k2') = ((16 - k1) mod 16, k1 ? 15 - k2 : (16 - k2) mod 16):
//   P = U_0[k1][k2] + W32^k2 U_1[k1][k2] = X[f],  P' = U_0 - W32^k2 U_1 = X[256 + f]
//   Q = U_0[k1'][k2'] -/+ W32^k2' U_1[k1'][k2'] = X[N - f],  the other sign X[256 - f]
// (the signs swap at f = 0, where the partner is the item itself).
template <int OUTK, int TP>
__device__ __forceinline__ void output_phase_512(const float2* __restrict__ U, const float2* __restrict__ tw,
                                                 const PipeArgs& a, int l, int64_t lm0, const float (&sw)[4],
                                                 void* __restrict__ qout, void* __restrict__ qlo) {
  constexpr int kOutCp = Geo<TP>::OUTCP, kItems = Geo<TP>::THREADS / kOutCp;
  const int cp = threadIdx.x % kOutCp;
  const float4* U4 = reinterpret_cast<const float4*>(U);
  const int64_t lm = lm0 + 4 * cp;
  // offset of row l at bin 0 and the step between bins (FP32 planar or BF16 blocked)
  constexpr bool BLK = OUTK != OUT_NATIVE;
  const int64_t o0 = BLK ? qhat_blocked_offset(a.nf, a.qrows, 0, l, lm) : (int64_t)l * a.chunk + lm;
  const int64_t fstep = BLK ? (int64_t)a.qrows * kQBlock : (int64_t)2 * a.nb * a.chunk;
  for (int j = threadIdx.x / kOutCp; j <= 128; j += kItems) {
    const int k1 = j & 15, k2 = j >> 4;
    const int k1p = (16 - k1) & 15;
    const int k2p = k1 ? 15 - k2 : (16 - k2) & 15;
    const float4 u0 = U4[(k1 * 16 + k2) * kOutCp + cp];
    const float4 u1 = c2mul(U4[((16 + k1) * 16 + k2) * kOutCp + cp], tw[16 * k2]);
    const float4 v0 = U4[(k1p * 16 + k2p) * kOutCp + cp];
    const float4 v1 = c2mul(U4[((16 + k1p) * 16 + k2p) * kOutCp + cp], tw[16 * k2p]);
    const float4 xf = c2add(u0, u1);                 // X[f]
    const float4 xf256 = c2sub(u0, u1);              // X[256 + f]
    const float4 xnf = j ? c2sub(v0, v1) : c2add(v0, v1);     // X[N - f]
    const float4 xg = j ? c2add(v0, v1) : c2sub(v0, v1);      // X[256 - f]
    store_bin4<OUTK>(xf, xnf, sw, a, o0 + j * fstep, qout, qlo);
    if (j != 128) store_bin4<OUTK>(xg, xf256, sw, a, o0 + (256 - j) * fstep, qout, qlo);
  }
}

// Shared-memory layout (bytes from the 1024-aligned base).
template <typename Tin, int TP, int N>
struct PipeLayout {
  static constexpr size_t hdr = 0;
  static constexpr size_t ring = 128;
  static constexpr size_t buf0 = ring + (size_t)N * TP * sizeof(Tin);
  static constexpr size_t buf1 = buf0 + (size_t)N * (TP / 2) * sizeof(float2);
  static constexpr size_t tw = buf1 + (size_t)N * (TP / 2) * sizeof(float2);
  static constexpr size_t win = tw + (size_t)N * sizeof(float2);
  // folded mean (kept out of the registers the passes need and of the pass
  // buffers): each thread's compensated sums of x - c, (s0, c0, s1, c1); the
  // threads' partial sums of the next tile's centre samples [32][TP]; the
  // centres and the rho values of a tile [TP] each; the centre sample rows
  static constexpr size_t acc = (win + (size_t)N * sizeof(float) + 15) / 16 * 16;
  static constexpr size_t cred = acc + (size_t)Geo<TP>::THREADS * sizeof(float4);
  static constexpr size_t cen = cred + (size_t)Geo<TP>::BSTEP * TP * sizeof(float);
  static constexpr size_t rho = cen + (size_t)TP * sizeof(float);
  static constexpr size_t crow = rho + (size_t)TP * sizeof(float);
  static constexpr size_t end = crow + (size_t)kCentreSamples * sizeof(int);
  static constexpr size_t dyn = end + 1024;                    // alignment slack
};

// 16-point tiles: two CTAs per SM up to nfft = 512 (shared memory allows it);
// otherwise one CTA gets the whole register file
template <int TP, int N> constexpr int pipe_min_blocks() { return TP == 16 && N <= 512 ? 2 : 1; }

template <typename Tin, int OUTK, int TP, int N, bool CPLX>
__global__ void __launch_bounds__(Geo<TP>::THREADS, pipe_min_blocks<TP, N>()) k_fft_pipe(const __grid_constant__ CUtensorMap xmap,
                                                          const float* __restrict__ win,
                                                          const float2* __restrict__ tw_g,
                                                          const float* __restrict__ sqrtW,
                                                          const double* __restrict__ mu, void* __restrict__ qout,
                                                          void* __restrict__ qlo, PipeArgs a,
                                                          unsigned* __restrict__ gflags) {
  using namespace tc;
  using L = PipeLayout<Tin, TP, N>;
  using S = PSeq<N>;
  constexpr int PTP = Geo<TP>::PTP, PC = Geo<TP>::PC, PTHREADS = Geo<TP>::THREADS;
  extern __shared__ unsigned char smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  PipeHdr* hdr = reinterpret_cast<PipeHdr*>(sm + L::hdr);
  Tin* ring = reinterpret_cast<Tin*>(sm + L::ring);
  float2* buf0 = reinterpret_cast<float2*>(sm + L::buf0);
  float2* buf1 = reinterpret_cast<float2*>(sm + L::buf1);
  float2* tw = reinterpret_cast<float2*>(sm + L::tw);
  float* wsm = reinterpret_cast<float*>(sm + L::win);
  const int tid = threadIdx.x;
  float4* const acc_all = reinterpret_cast<float4*>(sm + L::acc);
  float4* const my_acc = acc_all + tid;
  float* const cred = reinterpret_cast<float*>(sm + L::cred);
  float* const cen = reinterpret_cast<float*>(sm + L::cen);
  float* const rhos = reinterpret_cast<float*>(sm + L::rho);
  int* const crow = reinterpret_cast<int*>(sm + L::crow);
  const uint32_t bar = smem_u32(&hdr->full);
  volatile int* abort_flag = &hdr->abort;

  if (tid == 0) {
    mbar_init(bar, 1);
    hdr->abort = 0;
    fence_mbar_init();
  }
  for (int i = tid; i < N; i += PTHREADS) {
    tw[i] = tw_g[i];
    wsm[i] = win[i];
  }
  // folded mean: the centre's sample rows t_k = floor((2k + 1) nt / (2 nc))
  const int ncen = (int)(a.nt < kCentreSamples ? a.nt : kCentreSamples);
  if (tid < ncen) crow[tid] = (int)(((int64_t)(2 * tid + 1) * a.nt) / (2 * ncen));
  __syncthreads();

  const int64_t t_first = blockIdx.x;
  const int64_t t_step = gridDim.x;
  if (t_first >= a.ntiles) return;
  constexpr uint32_t row_bytes = PTP * sizeof(Tin);

  // TMA boxes for time rows [r0, r0 + nrows) of tile t; row r lands in ring slot r mod N
  auto issue = [&](int64_t t, int r0, int nrows) {
    mbar_arrive_expect_tx(bar, (uint32_t)nrows * row_bytes);
    const int x = (int)(a.m0 - a.xoff + t * PTP);
    for (int r = r0; r < r0 + nrows; r += a.boxr) tma_load_2d(smem_u32(ring + (size_t)(r % N) * PTP), &xmap, x, r, bar);
  };
  // L2 prefetch of time rows [r0, r0 + nrows) of tile t: the rows of block
  // l + 2 are requested from HBM while block l + 1's rows travel to the ring,
  // so the ring's load (one block ahead, all the shared memory allows) finds
  // them in L2
  auto prefetch = [&](int64_t t, int r0, int nrows) {
    const int x = (int)(a.m0 - a.xoff + t * PTP);
    for (int r = r0; r < r0 + nrows; r += a.boxr) tma_prefetch_2d(&xmap, x, r);
  };
  if (tid == 0) {
    prefetch_tmap(&xmap);
    issue(t_first, 0, N);
    if (a.nb > 1) prefetch(t_first, N, a.step);
  }

  const int col = tid % PC;
  uint32_t phase = 0;
  bool last_ok = true;               // thread 0: its last wait saw the copy land
  int par = 0;                       // buffer roles of the current block

  // Folded mean (real data, BF16 / BF16X3 output): the provisional centre c
  // of a column is the mean of its ncen snapshots at rows crow[k]; thread b of
  // a column sums k = b, b + 32, ...  The loads for tile t + t_step are issued
  // while tile t runs (pc0 / pc1) and reduced at its end.
  constexpr bool FOLDK = !CPLX && OUTK != OUT_NATIVE;
  const bool fold = FOLDK && a.fold;
  // real data at nfft = 512: the two-pass form (16 x 32, last radix 2 in the output phase)
  constexpr bool TWO = N == 512 && !CPLX;
  constexpr int PB = Geo<TP>::BSTEP;
  const int b0 = tid / PC;
  const Tin* const xg = static_cast<const Tin*>(a.xg);
  auto centre_partial = [&](int64_t t, float& c0, float& c1) {
    c0 = 0.f;
    c1 = 0.f;
    if (t >= a.ntiles) return;
    const int64_t lmA = t * PTP + 2 * col;
    const Tin* base = xg + a.xc0 + lmA;
#pragma unroll 1
    for (int k = b0; k < ncen; k += PB) {
      const Tin* row = base + (int64_t)crow[k] * a.xld;
      if (lmA < a.mcount) c0 += to_f32<Tin>(row[0]);
      if (lmA + 1 < a.mcount) c1 += to_f32<Tin>(row[1]);
    }
  };
  float cen0 = 0.f, cen1 = 0.f;      // this thread's column pair: centres of the current tile
  float pc0 = 0.f, pc1 = 0.f;        // partial centre sums of the next tile
  float swr = 0.f, cme = 0.f;        // threads < TP: sqrt(W) and centre of point tid of the tile
  if (fold) {
    centre_partial(t_first, pc0, pc1);
    cred[b0 * PTP + 2 * col] = pc0;
    cred[b0 * PTP + 2 * col + 1] = pc1;
    __syncthreads();
    if (tid < PTP) {
      float sm = 0.f;
#pragma unroll 1
      for (int q = 0; q < PB; ++q) sm += cred[q * PTP + tid];
      cen[tid] = sm / (float)ncen;
    }
    __syncthreads();
    cen0 = cen[2 * col];
    cen1 = cen[2 * col + 1];
    if (tid < PTP) cme = cen[tid];
    *my_acc = make_float4(0.f, 0.f, 0.f, 0.f);
    centre_partial(t_first + t_step, pc0, pc1);
  }
  for (int64_t t = t_first; t < a.ntiles; t += t_step) {
    const int64_t lm0 = t * PTP;
    const int64_t gm0 = a.m0 + lm0;
    float mhi0 = 0.f, mlo0 = 0.f, mhi1 = 0.f, mlo1 = 0.f;
    float sw[4];                     // 0.5 sqrt(W) of the output phase's four points (zero past mcount);
                                     // complex data: sqrt(W) of its two points
    {
      const int64_t lm = lm0 + 2 * col;
      if (a.subtract_mean && !a.fold && lm < a.mcount) {
        const double d = mu[gm0 + 2 * col]; mhi0 = (float)d; mlo0 = (float)(d - (double)mhi0);
      }
      if (a.subtract_mean && !a.fold && lm + 1 < a.mcount) {
        const double d = mu[gm0 + 2 * col + 1]; mhi1 = (float)d; mlo1 = (float)(d - (double)mhi1);
      }
      const int cp = tid % Geo<TP>::OUTCP;
      if constexpr (CPLX) {          // components -> points
        const int64_t lp = lm0 / 2 + 2 * cp, gp = gm0 / 2 + 2 * cp;
#pragma unroll
        for (int q = 0; q < 4; ++q) sw[q] = (q < 2 && 2 * (lp + q) < a.mcount) ? sqrtW[gp + q] : 0.f;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          sw[q] = (lm0 + 4 * cp + q < a.mcount) ? 0.5f * sqrtW[gm0 + 4 * cp + q] : 0.f;
      }
    }
    if (fold) {
      mhi0 = cen0;
      mhi1 = cen1;
      if (tid < PTP) swr = lm0 + tid < a.mcount ? sqrtW[gm0 + tid] : 0.f;
    }
    int rb = 0;                      // ring slot of the block's first row
    for (int l = 0; l < a.nb; ++l) {
      last_ok = mbar_wait(bar, phase & 1, abort_flag, gflags);
      ++phase;
      float2* bA = par ? buf1 : buf0;
      float2* bB = par ? buf0 : buf1;
      {
        // with the folded mean the centre c replaces mu (mlo = 0) and the
        // snapshots no earlier block held (all of block 0, the last step rows
        // of the others) are summed: FP32 runs of <= 16 samples, then a
        // compensated FP32 running sum
        // The new snapshots are n >= N - step; when N - step is a multiple of
        // N / R0 (50 % overlap, none, 75 %, ...) they are the elements
        // r >= (N - step) / (N / R0) of every first-pass butterfly, otherwise
        // a separate loop re-reads them from the ring.
        // (two-pass nfft = 512: the samples n1 >= (N - step) / 32 of pass A)
        constexpr int NBUT = TWO ? 32 : N / S::R0;
        constexpr int NGRP = TWO ? 16 : S::R0;
        const int nnew0 = !fold ? N : l == 0 ? 0 : N - a.step;
        const bool in_pass = nnew0 % NBUT == 0;
        const int rthr = fold && in_pass ? nnew0 / NBUT : NGRP;
        float s0 = 0.f, s1 = 0.f;
        if constexpr (TWO)
          pass_a512<Tin, TP, FOLDK>(ring, rb, bA, wsm, tw, mhi0, mlo0, mhi1, mlo1, rthr, s0, s1);
        else
          pass_first<Tin, TP, N, S::R0, FOLDK>(ring, rb, bA, wsm, mhi0, mlo0, mhi1, mlo1, rthr, s0, s1);
        if (fold) {
          if (!in_pass) {
            for (int n = nnew0 + tid / PC; n < N; n += Geo<TP>::BSTEP) {
              int slot = rb + n;
              if (slot >= N) slot -= N;
              const float2 x = PairLoad<Tin>::get(ring + slot * PTP + 2 * col);
              s0 += x.x - mhi0;
              s1 += x.y - mhi1;
            }
          }
          float4 ac = *my_acc;
          kahan_add(ac.x, ac.y, s0);
          kahan_add(ac.z, ac.w, s1);
          *my_acc = ac;
        }
      }
      __syncthreads();
      if (hdr->abort) break;
      // the ring rows of this block are consumed: request the next rows
      if (tid == 0) {
        if (l + 1 < a.nb) {
          issue(t, l * a.step + N, a.step);
          if (l + 2 < a.nb) prefetch(t, (l + 1) * a.step + N, a.step);   // rows of block l + 2 (< nt)
        } else if (t + t_step < a.ntiles) {
          issue(t + t_step, 0, N);
          if (a.nb > 1) prefetch(t + t_step, N, a.step);
        }
      }
      if constexpr (TWO) {
        // pass B writes bB, which the previous block's output phase read: every
        // thread has passed the barrier above since
        pass_b512<TP>(bA, bB);
        __syncthreads();
        output_phase_512<OUTK, TP>(bB, tw, a, l, lm0, sw, qout, qlo);
        // the next block's pass A writes bA, which nobody reads after pass B
      } else {
        const float2* spec = S::template rest<TP>(bA, bB, tw);
        if constexpr (CPLX) output_phase_cplx<OUTK, TP, N>(spec, a, l, lm0 / 2, sw, qout, qlo);
        else output_phase<OUTK, TP, N>(spec, a, l, lm0, sw, qout, qlo);
        par ^= (S::P & 1);
      }
      rb += a.step;
      if (rb >= N) rb -= N;
    }
    if (hdr->abort) break;
    if (fold) {
      // the snapshots in no block (the tail): thread b of a column takes t = tail0 + b + 32 k
      const int64_t lmA = lm0 + 2 * col;
      float4 ac = *my_acc;
      for (int64_t tt = a.tail0 + b0; tt < a.nt; tt += PB) {
        const Tin* row = xg + tt * a.xld + a.xc0 + lmA;
        if (lmA < a.mcount) kahan_add(ac.x, ac.y, to_f32<Tin>(row[0]) - mhi0);
        if (lmA + 1 < a.mcount) kahan_add(ac.z, ac.w, to_f32<Tin>(row[1]) - mhi1);
      }
      *my_acc = ac;
      cred[b0 * PTP + 2 * col] = pc0;
      cred[b0 * PTP + 2 * col + 1] = pc1;
      __syncthreads();
      if (tid < PTP) {
        // point tid: its column's 32 compensated partials in a fixed order,
        // mu = c + sum / nt, rho = sqrt(W) (mu - c)
        const int c = tid >> 1, h = tid & 1;
        float ss = 0.f, sc = 0.f, cc = 0.f;
#pragma unroll 1
        for (int q = 0; q < PB; ++q) {
          const float4 v = acc_all[q * PC + c];
          kahan_add(ss, sc, h ? v.z : v.x);
          cc += h ? v.w : v.y;
        }
        // each partial is s - c; the total (ss - sc) - sum of the c
        const double mup = ((double)ss - (double)sc - (double)cc) / (double)a.nt;
        float rho = 0.f;
        if (lm0 + tid < a.mcount) {
          a.mu_out[gm0 + tid] = (double)cme + mup;
          rho = (float)(mup * (double)swr);
        }
        rhos[tid] = rho;
      } else if (tid < 2 * PTP) {
        // the next tile's centre of point tid - TP
        const int p = tid - PTP;
        float sm = 0.f;
#pragma unroll 1
        for (int q = 0; q < PB; ++q) sm += cred[q * PTP + p];
        cen[p] = sm / (float)ncen;
      }
      __syncthreads();
      // rho into Qhat row 2 nb of every frequency (two points per word)
      for (int it = tid; it < a.nf * (PTP / 2); it += PTHREADS) {
        const int f = it / (PTP / 2), j = it - f * (PTP / 2);
        const int64_t o = qhat_blocked_offset(a.nf, a.qrows, f, 2 * a.nb, lm0 + 2 * j);
        const uint32_t hw = pack_bf16x2(rhos[2 * j], rhos[2 * j + 1]);
        *reinterpret_cast<uint32_t*>(static_cast<__nv_bfloat16*>(qout) + o) = hw;
        if constexpr (OUTK == OUT_BF16X3)
          *reinterpret_cast<uint32_t*>(static_cast<__nv_bfloat16*>(qlo) + o) =
              pack_bf16x2(rhos[2 * j] - bf16_lo_f(hw), rhos[2 * j + 1] - bf16_hi_f(hw));
      }
      cen0 = cen[2 * col];
      cen1 = cen[2 * col + 1];
      if (tid < PTP) cme = cen[tid];
      *my_acc = make_float4(0.f, 0.f, 0.f, 0.f);
      centre_partial(t + 2 * t_step, pc0, pc1);
      // cen and rhos are next written after the next tile's first barrier,
      // by which time every thread has read them
    }
  }
  // a request issued before an abort must land before the CTA exits
  if (tid == 0 && !last_ok) mbar_drain(bar, (phase - 1) & 1, gflags);
}

// Complex data (CPLX): m0 and mcount count points; the ring, the mean and the
// tiles work on the 2M interleaved components.
template <typename Tin, int OUTK, int TP, int N, bool CPLX>
cudaError_t launch_pipe_n(const spod_plan_s& p, const CUtensorMap& xmap, const void* d_X, int64_t m0,
                          int64_t mcount, cudaStream_t s) {
  constexpr int PTHREADS = Geo<TP>::THREADS;
  constexpr int64_t K = CPLX ? 2 : 1;          // components per point
  PipeArgs a;
  a.m0 = K * m0; a.mcount = K * mcount; a.chunk = p.chunk_points;
  a.xoff = K * p.x_off;
  const int64_t mpad = K * std::min<int64_t>(p.chunk_points, (mcount + 63) / 64 * 64);
  a.ntiles = mpad / TP;
  a.step = p.step; a.nb = p.nb; a.nf = p.nf;
  a.boxr = p.ring_boxr;
  a.subtract_mean = p.desc.subtract_mean;
  a.qrows = p.qrows;
  a.fold = (!CPLX && p.mean_fold) ? 1 : 0;
  a.nt = p.nt;
  a.tail0 = (int64_t)(p.nb - 1) * p.step + p.nfft;
  a.xg = d_X;
  a.xld = K * (p.x_ld ? p.x_ld : p.M);
  a.xc0 = a.m0 - a.xoff;
  a.mu_out = p.d_mu;
  const size_t smem = PipeLayout<Tin, TP, N>::dyn;
  auto kern = k_fft_pipe<Tin, OUTK, TP, N, CPLX>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PTHREADS, smem);
  per_sm = std::max(1, per_sm);
  const int grid = (int)std::min<int64_t>(a.ntiles, (int64_t)(p.num_sms > 0 ? p.num_sms : 148) * per_sm);
  if (grid <= 0) return cudaSuccess;
  kern<<<grid, PTHREADS, smem, s>>>(xmap, static_cast<const float*>(p.d_win), static_cast<const float2*>(p.d_tw),
                                    static_cast<const float*>(p.d_sqrtW), p.d_mu, p.d_qhat, p.d_qlo, a, p.d_flags);
  return cudaGetLastError();
}

template <typename Tin, int OUTK, bool CPLX>
cudaError_t launch_pipe_t(const spod_plan_s& p, const CUtensorMap& xmap, const void* d_X, int64_t m0,
                          int64_t mcount, cudaStream_t s) {
  if constexpr (sizeof(Tin) <= 4) {
    if (p.pipe_tp == 32) {
      switch (p.nfft) {
        case 256: return launch_pipe_n<Tin, OUTK, 32, 256, CPLX>(p, xmap, d_X, m0, mcount, s);
        case 384: return launch_pipe_n<Tin, OUTK, 32, 384, CPLX>(p, xmap, d_X, m0, mcount, s);
        case 512: return launch_pipe_n<Tin, OUTK, 32, 512, CPLX>(p, xmap, d_X, m0, mcount, s);
        default: return cudaErrorInvalidValue;
      }
    }
  }
  if (p.pipe_tp != 16) return cudaErrorInvalidValue;
  switch (p.nfft) {
    case 256: return launch_pipe_n<Tin, OUTK, 16, 256, CPLX>(p, xmap, d_X, m0, mcount, s);
    case 384: return launch_pipe_n<Tin, OUTK, 16, 384, CPLX>(p, xmap, d_X, m0, mcount, s);
    case 512: return launch_pipe_n<Tin, OUTK, 16, 512, CPLX>(p, xmap, d_X, m0, mcount, s);
    default: return launch_pipe_n<Tin, OUTK, 16, 720, CPLX>(p, xmap, d_X, m0, mcount, s);
  }
}

template <typename Tin, bool CPLX = false>
cudaError_t launch_pipe_in(const spod_plan_s& p, const CUtensorMap& xmap, const void* d_X, int64_t m0,
                           int64_t mcount, cudaStream_t s) {
  if (p.desc.precision == SPOD_PREC_BF16X3) return launch_pipe_t<Tin, OUT_BF16X3, CPLX>(p, xmap, d_X, m0, mcount, s);
  if (p.desc.precision == SPOD_PREC_BF16) return launch_pipe_t<Tin, OUT_BF16, CPLX>(p, xmap, d_X, m0, mcount, s);
  return launch_pipe_t<Tin, OUT_NATIVE, CPLX>(p, xmap, d_X, m0, mcount, s);
}

template <typename Tin, int TP>
size_t pipe_smem_t(int nfft) {
  switch (nfft) {
    case 256: return PipeLayout<Tin, TP, 256>::dyn;
    case 384: return PipeLayout<Tin, TP, 384>::dyn;
    case 512: return PipeLayout<Tin, TP, 512>::dyn;
    case 720:
      if constexpr (TP == 16) return PipeLayout<Tin, TP, 720>::dyn;
      return 0;
    default: return 0;
  }
}
template <typename Tin>
size_t pipe_smem_tp(int nfft, int tp) {
  if (tp == 32) {
    if constexpr (sizeof(Tin) <= 4) return pipe_smem_t<Tin, 32>(nfft);
    return 0;
  }
  return tp == 16 ? pipe_smem_t<Tin, 16>(nfft) : 0;
}

}  // namespace

// Dynamic shared memory of the pipelined kernel with tp-point tiles, 0 when
// nfft (or the input type) has no compiled form for that tile.
size_t fft_pipe_smem_bytes(const spod_plan_s& p, int tp) {
  switch (p.desc.in_dtype) {
    case SPOD_F64: case SPOD_C128: return pipe_smem_tp<double>(p.nfft, tp);
    case SPOD_F32: case SPOD_C64: return pipe_smem_tp<float>(p.nfft, tp);
    default: return pipe_smem_tp<__nv_bfloat16>(p.nfft, tp);
  }
}

// Tile width of the pipelined kernel: 32 points when that form exists and
// fits in shared memory, else 16.
int fft_pipe_tile(const spod_plan_s& p, int smem_optin) {
  const size_t s32 = fft_pipe_smem_bytes(p, 32);
  return s32 > 0 && s32 <= (size_t)smem_optin ? 32 : 16;
}

bool fft_pipe_usable(const spod_plan_s& p, int smem_optin) {
  if (p.f64 || p.ring_boxr <= 0) return false;
  const size_t el = p.desc.in_dtype == SPOD_F64 || p.desc.in_dtype == SPOD_C64 ? 8
                   : p.desc.in_dtype == SPOD_C128                              ? 16
                   : p.desc.in_dtype == SPOD_F32                               ? 4
                                                                               : 2;
  if ((p.M * (int64_t)el) % 16 != 0) return false;          // TMA row stride
  if (p.nfft % p.ring_boxr != 0 || p.step % p.ring_boxr != 0) return false;
  const size_t smem = fft_pipe_smem_bytes(p, p.pipe_tp);
  return smem > 0 && smem <= (size_t)smem_optin;
}

cudaError_t launch_fft_pipe_chunk(const spod_plan_s& p, const CUtensorMap& xmap, const void* d_X, int64_t m0,
                                  int64_t mcount, cudaStream_t s) {
  switch (p.desc.in_dtype) {
    case SPOD_F64: return launch_pipe_in<double>(p, xmap, d_X, m0, mcount, s);
    case SPOD_F32: return launch_pipe_in<float>(p, xmap, d_X, m0, mcount, s);
    case SPOD_C64: return launch_pipe_in<float, true>(p, xmap, d_X, m0, mcount, s);
    case SPOD_C128: return launch_pipe_in<double, true>(p, xmap, d_X, m0, mcount, s);
    default: return launch_pipe_in<__nv_bfloat16>(p, xmap, d_X, m0, mcount, s);
  }
}

}  // namespace spod
