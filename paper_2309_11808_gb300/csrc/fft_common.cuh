// Device helpers shared by the block-FFT kernels: complex arithmetic, the
// small forward DFTs of radix 2/3/4/5/8 and one Stockham pass.
#pragma once

#include "spod_internal.cuh"

namespace spod {
namespace fft {

template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

template <typename R> __device__ __forceinline__ typename C2<R>::T mk(R x, R y) {
  typename C2<R>::T v; v.x = x; v.y = y; return v;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { a.x += b.x; a.y += b.y; return a; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  V r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// multiply by -i
template <typename V> __device__ __forceinline__ V mul_mi(V a) { V r; r.x = a.y; r.y = -a.x; return r; }
template <typename V, typename R> __device__ __forceinline__ V cscale(V a, R s) { a.x *= s; a.y *= s; return a; }

template <typename T> __device__ __forceinline__ float to_f32(T v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float to_f32<double>(double v) { return (float)v; }

template <typename T> __device__ __forceinline__ double to_f64(T v) { return (double)to_f32<T>(v); }
template <> __device__ __forceinline__ double to_f64<double>(double v) { return v; }

// ---------------------------------------------------------------- FFT
struct FftArgs {
  int64_t M, m0, mcount, chunk;   // M = row stride of X in points; chunk = row stride of Qhat
  int64_t xoff;                   // point of X's first column (tiled data)
  int64_t mpad;                   // points written: mcount rounded up to 64 (zeros past mcount)
  int nfft, step, nb, nf;
  int qrows;                      // Qhat rows per frequency of the blocked layout
  int subtract_mean;
  FftPlan fp;
};

// R-point forward DFT in place, X_r = sum_q v_q exp(-2 pi i r q / R).
template <int RAD, typename V, typename R>
__device__ __forceinline__ void dft_small(V* v) {
  if constexpr (RAD == 2) {
    V a = v[0];
    v[0] = cadd(a, v[1]); v[1] = csub(a, v[1]);
  } else if constexpr (RAD == 3) {
    const R h = (R)0.86602540378443864676;   // sin(2 pi / 3)
    V s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    V m = mk<R>(v[0].x - (R)0.5 * s.x, v[0].y - (R)0.5 * s.y);
    V jd = mk<R>(h * d.y, -h * d.x);        // -i h d
    v[0] = cadd(v[0], s);
    v[1] = cadd(m, jd);
    v[2] = csub(m, jd);
  } else if constexpr (RAD == 4) {
    V a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    V c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
    v[0] = cadd(a, c); v[2] = csub(a, c);
    v[1] = cadd(b, mul_mi(d)); v[3] = csub(b, mul_mi(d));
  } else if constexpr (RAD == 5) {
    const R c1 = (R)0.30901699437494742410, c2 = (R)-0.80901699437494742410;
    const R s1 = (R)0.95105651629515357212, s2 = (R)0.58778525229247312917;
    V a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
    V a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
    V p1 = mk<R>(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
    V p2 = mk<R>(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
    V q1 = mk<R>(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y);   // X1 = p1 - i q1
    V q2 = mk<R>(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y);   // X2 = p2 - i q2
    v[0] = cadd(v[0], cadd(a1, a2));
    v[1] = cadd(p1, mul_mi(q1)); v[4] = csub(p1, mul_mi(q1));
    v[2] = cadd(p2, mul_mi(q2)); v[3] = csub(p2, mul_mi(q2));
  } else if constexpr (RAD == 8) {
    const R r2 = (R)0.70710678118654752440;
    V a[4], b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) { a[q] = cadd(v[q], v[q + 4]); b[q] = csub(v[q], v[q + 4]); }
    // b_q *= exp(-2 pi i q / 8)
    b[1] = mk<R>(r2 * (b[1].x + b[1].y), r2 * (b[1].y - b[1].x));
    b[2] = mul_mi(b[2]);
    b[3] = mk<R>(r2 * (b[3].y - b[3].x), -r2 * (b[3].x + b[3].y));
    dft_small<4, V, R>(a);
    dft_small<4, V, R>(b);
#pragma unroll
    for (int k = 0; k < 4; ++k) { v[2 * k] = a[k]; v[2 * k + 1] = b[k]; }
  }
}

// One Stockham pass of radix RAD over C interleaved sequences of length n
// (layout [n][C]) from src to dst.  Butterfly b uses k = b mod Ns and group
// b / Ns; the power-of-two passes run first, so Ns stays a power of two
// (shift and mask) until the radix-3/5 passes.  C is a compile-time constant.
template <int RAD, int C, typename V, typename R>
__device__ __forceinline__ void stockham_pass(const V* __restrict__ src, V* __restrict__ dst,
                                              const V* __restrict__ tw, int n, int Ns, int log2Ns) {
  const int nbut = n / RAD;
  const int stride_tw = n / (Ns * RAD);
  for (int idx = threadIdx.x; idx < nbut * C; idx += blockDim.x) {
    const int b = idx / C, col = idx % C;
    V v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[r] = src[(b + r * nbut) * C + col];
    int k, g;
    if (log2Ns >= 0) { k = b & (Ns - 1); g = b >> log2Ns; }
    else { g = b / Ns; k = b - g * Ns; }
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < RAD; ++r) v[r] = cmul(v[r], tw[r * k * stride_tw]);
    }
    dft_small<RAD, V, R>(v);
    const int base = g * Ns * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) dst[(base + r * Ns) * C + col] = v[r];
  }
}

// Output element types of the FFT kernel.
enum OutKind { OUT_NATIVE = 0, OUT_BF16X3 = 1, OUT_BF16 = 2 };


}  // namespace fft
}  // namespace spod
