// Weighted cross-spectral Gram of the method of snapshots
// (Eq. spod-discrete-snapshots): M_f = kappa * Qhat_f^* W Qhat_f, computed in
// SIMT arithmetic (FP32 or FP64) from the planar Qhat written by the FFT
// kernel (sqrt(W) already folded in).
//
// Grid: (split s, frequency f).  Each CTA owns a contiguous range of the
// chunk's points and one thread per 4x4 tile of the upper triangle of the
// nb x nb complex Gram.  FP32 partial sums are promoted to FP64 every kFlush
// points.  Partials are kept per split in FP64 and added chunk after chunk in
// stream order, then summed over splits in a fixed order by k_gram_reduce:
// no atomics, so the result is bit-reproducible (the in-GPU counterpart of
// the paper's single reduction of the Gram over ranks, Sec. 3.1).
#include "spod_internal.cuh"

namespace spod {
namespace {

constexpr int TK = 32;        // points staged per step
constexpr int kFlush = 256;   // FP32 -> FP64 promotion interval (points)

__device__ __forceinline__ void load4(const float* p, float* v) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void load4(const double* p, double* v) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

template <typename R>
__global__ void __launch_bounds__(256) k_gram_simt(const R* __restrict__ qhat, int64_t rs, int nb, int64_t mcount,
                                                   int64_t per_split, int first, double* __restrict__ gpart,
                                                   int nf) {
  const int s = blockIdx.x;
  const int f = blockIdx.y;
  const int ntl = (nb + 3) / 4;
  const int RS = 4 * ntl;                       // staged row stride (rows padded with zeros)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sR = reinterpret_cast<R*>(smem_raw);       // [TK][RS]
  R* sI = sR + TK * RS;                         // [TK][RS]

  // this thread's tile (I <= J) of the upper triangle; grid.z splits the tiles
  const int ntiles = ntl * (ntl + 1) / 2;
  const int tix = blockIdx.z * blockDim.x + threadIdx.x;
  int I = 0, J = 0;
  const bool active = tix < ntiles;
  {
    int t = tix, row = 0;
    while (active && t >= ntl - row) { t -= ntl - row; ++row; }
    I = row; J = row + t;
  }

  const int64_t p0 = (int64_t)s * per_split;
  const int64_t p1 = min(mcount, p0 + per_split);
  const R* qf = qhat + (int64_t)f * 2 * nb * rs;

  R ar[4][4], ai[4][4];
  double dr[4][4], di[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { ar[i][j] = 0; ai[i][j] = 0; dr[i][j] = 0; di[i][j] = 0; }

  int since_flush = 0;
  for (int64_t pb = p0; pb < p1; pb += TK) {
    __syncthreads();
    // stage rows (re: 0..nb-1, im: nb..2nb-1) of points [pb, pb+TK)
    for (int idx = threadIdx.x; idx < 2 * RS * TK; idx += blockDim.x) {
      const int row = idx / TK, k = idx - row * TK;
      const int c = row / RS, l = row - c * RS;
      R v = 0;
      if (l < nb && pb + k < p1) v = qf[((int64_t)c * nb + l) * rs + pb + k];
      (c == 0 ? sR : sI)[k * RS + l] = v;
    }
    __syncthreads();
    if (active) {
      const int kmax = (int)min((int64_t)TK, p1 - pb);
      for (int k = 0; k < kmax; ++k) {
        R xr[4], xi[4], yr[4], yi[4];
        // 4-wide shared loads (rows are padded to a multiple of 4)
        load4(sR + k * RS + 4 * I, xr);
        load4(sI + k * RS + 4 * I, xi);
        load4(sR + k * RS + 4 * J, yr);
        load4(sI + k * RS + 4 * J, yi);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            // conj(x_i) * y_j
            ar[i][j] += xr[i] * yr[j] + xi[i] * yi[j];
            ai[i][j] += xr[i] * yi[j] - xi[i] * yr[j];
          }
      }
      since_flush += kmax;
      if (sizeof(R) == 4 && since_flush >= kFlush) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            dr[i][j] += (double)ar[i][j]; di[i][j] += (double)ai[i][j];
            ar[i][j] = 0; ai[i][j] = 0;
          }
        since_flush = 0;
      }
    }
  }
  if (!active) return;
  double* g = gpart + (((int64_t)s * nf + f) * nb) * nb * 2;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int li = 4 * I + i, lj = 4 * J + j;
      if (li >= nb || lj >= nb || lj < li) continue;
      const double vr = dr[i][j] + (double)ar[i][j];
      const double vi = di[i][j] + (double)ai[i][j];
      double* e = g + ((int64_t)li * nb + lj) * 2;
      if (first) { e[0] = vr; e[1] = vi; }
      else { e[0] += vr; e[1] += vi; }
    }
}

// Fixed-order sum over splits, kappa, Hermitian completion, NaN check.
__global__ void k_gram_reduce(const double* __restrict__ gpart, int splits, int nf, int nb, double kappa,
                              double* __restrict__ gram, unsigned* __restrict__ flags) {
  const int f = blockIdx.x;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e - i * nb;
    const int a = min(i, j), b = max(i, j);
    double vr = 0.0, vi = 0.0;
    for (int s = 0; s < splits; ++s) {
      const double* src = gpart + ((((int64_t)s * nf + f) * nb + a) * nb + b) * 2;
      vr += src[0]; vi += src[1];
    }
    vr *= kappa; vi *= kappa;
    if (i > j) vi = -vi;
    if (i == j) {
      vi = 0.0;
      if (!isfinite(vr)) atomicOr(flags, FLAG_NAN);
    }
    double* dst = gram + (((int64_t)f * nb + i) * nb + j) * 2;
    dst[0] = vr; dst[1] = vi;
  }
}

template <typename R>
cudaError_t launch_gram_t(const spod_plan_s& p, int64_t mcount, bool first, cudaStream_t s) {
  const int ntl = (p.nb + 3) / 4;
  const int ntiles = ntl * (ntl + 1) / 2;
  const int threads = min(256, max(32, ((ntiles + 31) / 32) * 32));
  const int groups = (ntiles + threads - 1) / threads;
  const size_t smem = 2 * (size_t)TK * 4 * ntl * sizeof(R);
  auto kern = k_gram_simt<R>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t per = (mcount + p.gram_splits - 1) / p.gram_splits;
  per = ((per + TK - 1) / TK) * TK;
  dim3 grid((unsigned)p.gram_splits, (unsigned)p.nf, (unsigned)groups);
  kern<<<grid, threads, smem, s>>>(static_cast<const R*>(p.d_qhat), p.chunk_points, p.nb, mcount, per,
                                   first ? 1 : 0, p.d_gpart, p.nf);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gram_chunk(const spod_plan_s& p, int64_t mcount, bool first, cudaStream_t s) {
  return p.f64 ? launch_gram_t<double>(p, mcount, first, s) : launch_gram_t<float>(p, mcount, first, s);
}

cudaError_t launch_gram_reduce(const spod_plan_s& p, cudaStream_t s) {
  k_gram_reduce<<<p.nf, 256, 0, s>>>(p.d_gpart, p.gram_splits, p.nf, p.nb, p.kappa, p.d_gram, p.d_flags);
  return cudaGetLastError();
}

}  // namespace spod
