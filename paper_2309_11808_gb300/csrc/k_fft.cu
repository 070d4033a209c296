// Time mean (Sec. 2.2) and the batched windowed block DFT (Eqs. blocks,
// blocks-ft, blocks-k) of the SPOD hot path.
//
// Mean: FP64 accumulation of FP32 runs of 16 samples (FP64 throughout for FP64
// input), time axis split over grid.y, then a fixed-order FP64 sum.
//
// FFT: one CTA of 256 threads per (Welch block l, tile of TP spatial points;
// TP = 16 for FP32 arithmetic, 8 for FP64).  Two real point series are
// packed into one complex sequence (z = x_even + i x_odd), the tile's TP/2
// sequences are transformed together by a shared-memory Stockham FFT of mixed
// radix 8/4/2/3/5 (ping-pong buffers, nfft <= 1024), and the two real spectra
// are separated at the end.  The mean is subtracted as a double-float pair, the window carries
// c = 1/sum(w), and sqrt(W_m) is folded into the output so that the Gram is a
// plain Qhat^H Qhat.  Output: Qhat[f][row][m_local], row = l (real part) or
// nb + l (imaginary part), f = 0 .. nfft/2.
#include <algorithm>

#include "fft_common.cuh"

namespace spod {
namespace {

using namespace fft;

// ---------------------------------------------------------------- mean
// part[y][m] (row stride M) sums rows [y tper, (y+1) tper) of column m of X,
// whose rows are xld columns long and start at column xoff.
template <typename Tin>
__global__ void __launch_bounds__(256) k_mean_partial(const Tin* __restrict__ X, int64_t M, int64_t xld, int64_t xoff,
                                                      int64_t nt, int64_t tper, int64_t m0, int64_t m1,
                                                      double* __restrict__ part) {
  const int64_t m = m0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= m1) return;
  const int64_t t0 = (int64_t)blockIdx.y * tper;
  const int64_t t1 = min(nt, t0 + tper);
  double acc = 0.0;
  const int64_t Mx = xld;                      // row stride of X
  const Tin* p = X + t0 * Mx + (m - xoff);
  int64_t t = t0;
  if constexpr (sizeof(Tin) == 8) {
    for (; t < t1; ++t, p += Mx) acc += (double)(*p);
  } else {
    for (; t + 16 <= t1; t += 16) {
      float r = 0.f;
#pragma unroll
      for (int i = 0; i < 16; ++i) r += to_f32<Tin>(p[i * Mx]);
      acc += (double)r;
      p += 16 * Mx;
    }
    for (; t < t1; ++t, p += Mx) acc += (double)to_f32<Tin>(*p);
  }
  part[(int64_t)blockIdx.y * M + m] = acc;
}

__global__ void k_mean_finish(const double* __restrict__ part, int splits, int64_t M, int64_t m0, int64_t m1,
                              double inv_nt, double* __restrict__ mu) {
  const int64_t m = m0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= m1) return;
  double s = 0.0;
  for (int i = 0; i < splits; ++i) s += part[(int64_t)i * M + m];
  mu[m] = s * inv_nt;
}

// One CTA (256 threads) per (Welch block l, tile of TP points).  Real data:
// two points share each of the TP/2 complex columns and are separated after
// the transform.  Complex data (CPLX; X holds interleaved real, imaginary
// components of type Tin): one point per column, TP/2 points per tile, and
// every one of the nfft bins is kept.
template <typename Tin, typename R, int TP, int OUTK, bool CPLX = false>
__global__ void __launch_bounds__(256) k_fft(const Tin* __restrict__ X, const R* __restrict__ win,
                                             const typename C2<R>::T* __restrict__ tw_g,
                                             const R* __restrict__ sqrtW, const double* __restrict__ mu,
                                             void* __restrict__ qout, void* __restrict__ qout_lo, FftArgs a) {
  using V = typename C2<R>::T;
  constexpr int C = TP / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* bufA = reinterpret_cast<V*>(smem_raw);
  V* bufB = bufA + (size_t)a.nfft * C;
  V* tw = bufB + (size_t)a.nfft * C;
  const int N = a.nfft;

  const int64_t item = blockIdx.x;
  const int l = (int)(item % a.nb);
  const int64_t tile = item / a.nb;
  constexpr int PPT = CPLX ? TP / 2 : TP; // points per tile
  const int64_t lm0 = tile * PPT;         // local (chunk) point index
  const int64_t gm0 = a.m0 + lm0;         // global point index

  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];

  // ---- load block l: thread owns column pair j, rows n = n0, n0 + 256/C, ...
  // (the mean is read once per column and kept as a rounded pair hi + lo)
  {
    // the column's two real values: points m, m + 1 (real data) or the real
    // and imaginary parts of point m (complex data), both at component index xi
    const int j = threadIdx.x % C;
    const int n0 = threadIdx.x / C;
    const int64_t m = gm0 + (CPLX ? j : 2 * j);
    const int64_t xi = CPLX ? 2 * m : m;          // mean (global)
    const int64_t xc = CPLX ? 2 * (m - a.xoff) : m - a.xoff;   // column of X
    const int64_t mend = a.m0 + a.mcount;
    const bool ok0 = m < mend, ok1 = CPLX ? ok0 : m + 1 < mend;
    R mhi0 = 0, mlo0 = 0, mhi1 = 0, mlo1 = 0;
    if (a.subtract_mean) {
      if (ok0) { const double d = mu[xi]; mhi0 = (R)d; mlo0 = (R)(d - (double)mhi0); }
      if (ok1) { const double d = mu[xi + 1]; mhi1 = (R)d; mlo1 = (R)(d - (double)mhi1); }
    }
    const int64_t rowlen = CPLX ? 2 * a.M : a.M;   // components per snapshot
    const Tin* base = X + (int64_t)l * a.step * rowlen + xc;
    constexpr int NSTEP = 256 / C;
#pragma unroll 4
    for (int n = n0; n < N; n += NSTEP) {
      const Tin* row = base + (int64_t)n * rowlen;
      R x0 = ok0 ? (R)to_f64<Tin>(row[0]) : (R)0;
      R x1 = ok1 ? (R)to_f64<Tin>(row[1]) : (R)0;
      x0 = ok0 ? (x0 - mhi0) - mlo0 : (R)0;
      x1 = ok1 ? (x1 - mhi1) - mlo1 : (R)0;
      const R wn = win[n];
      bufA[n * C + j] = mk<R>(x0 * wn, x1 * wn);
    }
  }
  __syncthreads();

  V* src = bufA;
  V* dst = bufB;
  int Ns = 1, log2Ns = 0;
  for (int ps = 0; ps < a.fp.npass; ++ps) {
    const int rad = a.fp.radix[ps];
    switch (rad) {
      case 8: stockham_pass<8, C, V, R>(src, dst, tw, N, Ns, log2Ns); break;
      case 4: stockham_pass<4, C, V, R>(src, dst, tw, N, Ns, log2Ns); break;
      case 2: stockham_pass<2, C, V, R>(src, dst, tw, N, Ns, log2Ns); break;
      case 3: stockham_pass<3, C, V, R>(src, dst, tw, N, Ns, log2Ns); break;
      default: stockham_pass<5, C, V, R>(src, dst, tw, N, Ns, log2Ns); break;
    }
    Ns *= rad;
    if (log2Ns >= 0) log2Ns = (rad == 2) ? log2Ns + 1 : (rad == 4) ? log2Ns + 2 : (rad == 8) ? log2Ns + 3 : -1;
    __syncthreads();
    V* t = src; src = dst; dst = t;
  }
  V* buf = src;

  // ---- separate the two real spectra, fold sqrt(W), store planar re/im rows;
  // points past mcount (up to the 64-point padding) are written as zeros
  const int64_t rs = a.chunk;
  for (int idx = threadIdx.x; idx < a.nf * PPT; idx += blockDim.x) {
    const int f = idx / PPT, p = idx - f * PPT;
    const int64_t lm = lm0 + p;
    if (lm >= a.mpad) continue;
    R re = 0, im = 0;
    if (lm < a.mcount) {
      if constexpr (CPLX) {          // column p is point p: Z[f] as it is
        const V z = buf[f * C + p];
        re = z.x;
        im = z.y;
      } else {
        const int col = p >> 1;
        const V zf = buf[f * C + col];
        const int fn = (f == 0) ? 0 : N - f;
        const V zc = buf[fn * C + col];
        if ((p & 1) == 0) {          // (Z[f] + conj Z[N-f]) / 2
          re = (R)0.5 * (zf.x + zc.x);
          im = (R)0.5 * (zf.y - zc.y);
        } else {                     // (Z[f] - conj Z[N-f]) / (2i)
          re = (R)0.5 * (zf.y + zc.y);
          im = (R)-0.5 * (zf.x - zc.x);
        }
      }
      const R sw = sqrtW[gm0 + p];
      re *= sw;
      im *= sw;
    }
    // planar FP32/FP64 rows, or 64-point blocked BF16 rows (qhat_blocked_offset)
    const int64_t o_re = (OUTK == OUT_NATIVE) ? ((int64_t)f * 2 * a.nb + l) * rs + lm
                                              : qhat_blocked_offset(a.nf, a.qrows, f, l, lm);
    const int64_t o_im = o_re + (int64_t)a.nb * ((OUTK == OUT_NATIVE) ? rs : (int64_t)kQBlock);
    if constexpr (OUTK == OUT_NATIVE) {
      R* q = static_cast<R*>(qout);
      q[o_re] = re;
      q[o_im] = im;
    } else {
      __nv_bfloat16* qh = static_cast<__nv_bfloat16*>(qout);
      const __nv_bfloat16 hr = __float2bfloat16_rn((float)re), hi = __float2bfloat16_rn((float)im);
      qh[o_re] = hr;
      qh[o_im] = hi;
      if constexpr (OUTK == OUT_BF16X3) {
        __nv_bfloat16* ql = static_cast<__nv_bfloat16*>(qout_lo);
        ql[o_re] = __float2bfloat16_rn((float)re - __bfloat162float(hr));
        ql[o_im] = __float2bfloat16_rn((float)im - __bfloat162float(hi));
      }
    }
  }
}

template <typename Tin, typename R, int OUTK, bool CPLX = false>
cudaError_t launch_fft_t(const spod_plan_s& p, const void* d_X, int64_t m0, int64_t mcount, cudaStream_t s) {
  constexpr int TP = sizeof(R) == 8 ? 8 : 16;
  constexpr int PPT = CPLX ? TP / 2 : TP;
  FftArgs a;
  a.M = p.x_ld ? p.x_ld : p.M; a.xoff = p.x_off; a.m0 = m0; a.mcount = mcount; a.chunk = p.chunk_points;
  a.mpad = std::min<int64_t>(p.chunk_points, (mcount + 63) / 64 * 64);
  a.nfft = p.nfft; a.step = p.step; a.nb = p.nb; a.nf = p.nf;
  a.qrows = p.qrows;
  a.subtract_mean = p.desc.subtract_mean;
  a.fp = p.fft;
  const size_t smem = fft_smem_bytes(p);
  auto kern = k_fft<Tin, R, TP, OUTK, CPLX>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (a.mpad + PPT - 1) / PPT;
  const int64_t grid = ntiles * p.nb;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  kern<<<(unsigned)grid, 256, smem, s>>>(
      static_cast<const Tin*>(d_X), static_cast<const R*>(p.d_win),
      static_cast<const typename C2<R>::T*>(p.d_tw), static_cast<const R*>(p.d_sqrtW), p.d_mu,
      p.d_qhat, p.d_qlo, a);
  return cudaGetLastError();
}

template <typename Tin>
// Mean of the real columns [m0, m0 + mcount) of a [nt][Mcols] array.
cudaError_t launch_mean_t(const spod_plan_s& p, const void* d_X, int64_t Mcols, int64_t m0, int64_t mcount,
                          cudaStream_t s) {
  const int64_t tper = (p.nt + p.mean_splits - 1) / p.mean_splits;
  const int64_t k = Mcols / p.M;              // 2 for complex data (components)
  const int64_t xld = k * (p.x_ld ? p.x_ld : p.M), xoff = k * p.x_off;
  dim3 grid((unsigned)((mcount + 255) / 256), (unsigned)p.mean_splits);
  k_mean_partial<Tin><<<grid, 256, 0, s>>>(static_cast<const Tin*>(d_X), Mcols, xld, xoff, p.nt, tper, m0,
                                           m0 + mcount, p.d_mupart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_mean_finish<<<(unsigned)((mcount + 255) / 256), 256, 0, s>>>(p.d_mupart, p.mean_splits, Mcols, m0,
                                                                  m0 + mcount, 1.0 / (double)p.nt, p.d_mu);
  return cudaGetLastError();
}

}  // namespace

size_t fft_smem_bytes(const spod_plan_s& p) {
  const size_t vb = p.f64 ? 16 : 8;
  const size_t C = p.f64 ? 4 : 8;
  return vb * ((size_t)p.nfft * C * 2 + (size_t)p.nfft);
}

cudaError_t launch_mean(const spod_plan_s& p, const void* d_X, int64_t m0, int64_t mcount, cudaStream_t s) {
  if (mcount <= 0) return cudaSuccess;
  switch (p.desc.in_dtype) {
    case SPOD_F64: return launch_mean_t<double>(p, d_X, p.M, m0, mcount, s);
    case SPOD_F32: return launch_mean_t<float>(p, d_X, p.M, m0, mcount, s);
    // complex data: the real and imaginary parts are 2M interleaved real columns
    case SPOD_C64: return launch_mean_t<float>(p, d_X, 2 * p.M, 2 * m0, 2 * mcount, s);
    case SPOD_C128: return launch_mean_t<double>(p, d_X, 2 * p.M, 2 * m0, 2 * mcount, s);
    default: return launch_mean_t<__nv_bfloat16>(p, d_X, p.M, m0, mcount, s);
  }
}

template <typename Tin, bool CPLX = false>
static cudaError_t launch_fft_in(const spod_plan_s& p, const void* d_X, int64_t m0, int64_t mcount, cudaStream_t s) {
  if (p.f64) return launch_fft_t<Tin, double, OUT_NATIVE, CPLX>(p, d_X, m0, mcount, s);
  if (p.desc.precision == SPOD_PREC_BF16X3) return launch_fft_t<Tin, float, OUT_BF16X3, CPLX>(p, d_X, m0, mcount, s);
  if (p.desc.precision == SPOD_PREC_BF16) return launch_fft_t<Tin, float, OUT_BF16, CPLX>(p, d_X, m0, mcount, s);
  return launch_fft_t<Tin, float, OUT_NATIVE, CPLX>(p, d_X, m0, mcount, s);
}

cudaError_t launch_fft_chunk(const spod_plan_s& p, const void* d_X, int64_t m0, int64_t mcount,
                             cudaStream_t s) {
  switch (p.desc.in_dtype) {
    case SPOD_F64: return launch_fft_in<double>(p, d_X, m0, mcount, s);
    case SPOD_F32: return launch_fft_in<float>(p, d_X, m0, mcount, s);
    case SPOD_C64: return launch_fft_in<float, true>(p, d_X, m0, mcount, s);
    case SPOD_C128: return launch_fft_in<double, true>(p, d_X, m0, mcount, s);
    default: return launch_fft_in<__nv_bfloat16>(p, d_X, m0, mcount, s);
  }
}

bool make_fft_plan(int n, FftPlan* fp) {
  fp->n = n;
  fp->npass = 0;
  int r = n;
  while (r % 8 == 0 && fp->npass < kMaxRadixPasses) { fp->radix[fp->npass++] = 8; r /= 8; }
  while (r % 4 == 0 && fp->npass < kMaxRadixPasses) { fp->radix[fp->npass++] = 4; r /= 4; }
  while (r % 2 == 0 && fp->npass < kMaxRadixPasses) { fp->radix[fp->npass++] = 2; r /= 2; }
  while (r % 3 == 0 && fp->npass < kMaxRadixPasses) { fp->radix[fp->npass++] = 3; r /= 3; }
  while (r % 5 == 0 && fp->npass < kMaxRadixPasses) { fp->radix[fp->npass++] = 5; r /= 5; }
  return r == 1;
}

}  // namespace spod
