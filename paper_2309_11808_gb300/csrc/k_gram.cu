// Weighted cross-spectral Gram of the method of snapshots
// (Eq. spod-discrete-snapshots): M_f = kappa * Qhat_f^* W Qhat_f, computed in
// SIMT arithmetic (FP32 or FP64) from the planar Qhat written by the FFT
// kernel (sqrt(W) already folded in).
//
// Grid: (split s, frequency f, tile group).  Each CTA owns a contiguous range
// of the chunk's points; four groups of 64 threads share it point by point,
// one thread per 4x4 tile of the upper triangle of the nb x nb complex Gram
// in each group.  FP32 partial sums are promoted to FP64 every 512 points of
// a thread (FP64 sums stay in registers).  Partials are kept per split in FP64 and added chunk after chunk in
// stream order, then summed over splits in a fixed order by k_gram_reduce:
// no atomics, so the result is bit-reproducible (the in-GPU counterpart of
// the paper's single reduction of the Gram over ranks, Sec. 3.1).
#include <algorithm>

#include "spod_internal.cuh"

namespace spod {
namespace {

constexpr int TK = 32;        // points staged per round
constexpr int KSUB = 4;       // thread groups splitting a round's points (point k goes to group k % KSUB)
constexpr int TPG = 64;       // threads per group: one 4x4 complex tile of the upper triangle each
constexpr int kThreads = KSUB * TPG;
// FP32 -> FP64 promotion every 64 rounds (TK * 64 / KSUB = 512 points a
// thread): FP64 adds issue at a small fraction of the FP32 rate on this part,
// so the promotion is kept rare; round-to-nearest FP32 runs of 512 products
// keep the partial sums to ~sqrt(512) 2^-24 relative
constexpr int kFlushRounds = 64;
constexpr size_t kGramSimtSmemMax = 227 * 1024;

// Staged row stride: the row quads of a point padded to an odd count, so the
// 16-byte staging stores of eight consecutive points (one shared-memory
// phase) start in eight distinct groups of four banks.
__host__ __device__ constexpr int staged_stride(int nb) { return 4 * (((nb + 3) / 4) | 1); }

__device__ __forceinline__ void store4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(double* p, const double* v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// 4-wide shared loads (rows are padded to a multiple of 4)
__device__ __forceinline__ void load4(const float* p, float* v) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void load4(const double* p, double* v) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// One CTA per (split of the chunk's points, frequency, group of 64 tiles).
// Rounds of TK points are staged (transposed, [point][row]) into nbuf shared
// buffers: the next round's global loads are issued before the current round
// is used, and stored after it (into the other buffer, or into the same one
// after a barrier when only one fits).  Thread (group q, tile t) accumulates
// tile t over the round's points k = q, q + KSUB, ...; FP32 partial sums are
// added into FP64 sums in shared memory every kFlushRounds rounds, and the
// KSUB groups' FP64 sums are combined in group order at the end (for FP64 the
// combining area overlays the staging buffers, which are idle by then).
template <typename R>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 2 : 1) k_gram_simt(const R* __restrict__ qhat, int64_t rs, int nb,
                                                           int64_t mcount, int64_t per_split, int first, int nbuf,
                                                           double* __restrict__ gpart, int nf) {
  constexpr bool kPromote = sizeof(R) == 4;
  const int s = blockIdx.x;
  const int f = blockIdx.y;
  const int ntl = (nb + 3) / 4;
  const int RS = staged_stride(nb);             // staged row stride (rows padded with zeros)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* acc64 = reinterpret_cast<double*>(smem_raw);             // [32][kThreads]
  R* stage = kPromote ? reinterpret_cast<R*>(acc64 + 32 * kThreads)  // [nbuf][re, im][TK][RS]
                      : reinterpret_cast<R*>(smem_raw);
  const int buf_elems = 2 * TK * RS;

  const int tid = threadIdx.x;
  const int q = tid / TPG;
  const int ntiles = ntl * (ntl + 1) / 2;
  const int tix = blockIdx.z * TPG + (tid % TPG);
  int I = 0, J = 0;
  const bool active = tix < ntiles;
  {
    int t = tix, row = 0;
    while (active && t >= ntl - row) { t -= ntl - row; ++row; }
    I = row; J = row + t;
  }
  if (kPromote) {
#pragma unroll
    for (int e = 0; e < 32; ++e) acc64[e * kThreads + tid] = 0.0;
  }

  const int64_t p0 = (int64_t)s * per_split;
  const int64_t p1 = min(mcount, p0 + per_split);
  const R* qf = qhat + (int64_t)f * 2 * nb * rs;
  const int nrounds = p1 > p0 ? (int)((p1 - p0 + TK - 1) / TK) : 0;

  // staging: item e of a round = (plane c, row quad u, point k), point
  // fastest: each thread loads the quad's four rows at its point (coalesced
  // over the warp's points) and stores them as one 16-byte (FP64: two)
  // shared store at [c][k][4u].  Items past the prefetched ones (nb > 64) are
  // copied directly.
  const int nq = 2 * ntl;                       // row quads of both planes
  constexpr int kMaxItems = (2 * 16 * TK + kThreads - 1) / kThreads;
  R pre[kMaxItems][4];
  auto item = [&](int it, int& k, int& c, int& u) {
    k = it % TK;
    const int qd = it / TK;
    c = qd >= ntl ? 1 : 0;
    u = qd - c * ntl;
    return qd < nq;
  };
  auto fetch = [&](int r) {
    const int64_t pb = p0 + (int64_t)r * TK;
#pragma unroll
    for (int j = 0; j < kMaxItems; ++j) {
      int k, c, u;
      const bool in = item(tid + j * kThreads, k, c, u) && pb + k < p1;
      const R* src = qf + pb + k;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int l = 4 * u + e;
        pre[j][e] = (in && l < nb) ? src[((int64_t)c * nb + l) * rs] : R(0);
      }
    }
  };
  auto put = [&](int b, int r) {
    R* st = stage + b * buf_elems;
#pragma unroll
    for (int j = 0; j < kMaxItems; ++j) {
      int k, c, u;
      if (item(tid + j * kThreads, k, c, u)) store4(st + c * TK * RS + k * RS + 4 * u, pre[j]);
    }
    const int64_t pb = p0 + (int64_t)r * TK;
    for (int it = kMaxItems * kThreads + tid; it < nq * TK; it += kThreads) {
      int k, c, u;
      item(it, k, c, u);
      R v[4];
      for (int e = 0; e < 4; ++e) {
        const int l = 4 * u + e;
        v[e] = (l < nb && pb + k < p1) ? qf[((int64_t)c * nb + l) * rs + pb + k] : R(0);
      }
      store4(st + c * TK * RS + k * RS + 4 * u, v);
    }
  };

  R ar[4][4], ai[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { ar[i][j] = 0; ai[i][j] = 0; }
  auto flush = [&]() {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        double* er = acc64 + (2 * (4 * i + j)) * kThreads + tid;
        double* ei = er + kThreads;
        if (kPromote) { *er += (double)ar[i][j]; *ei += (double)ai[i][j]; }
        else { *er = (double)ar[i][j]; *ei = (double)ai[i][j]; }
        ar[i][j] = 0; ai[i][j] = 0;
      }
  };

  if (nrounds > 0) {
    fetch(0);
    put(0, 0);
  }
  __syncthreads();
  for (int r = 0; r < nrounds; ++r) {
    const int b = nbuf == 2 ? (r & 1) : 0;
    if (r + 1 < nrounds) fetch(r + 1);        // in flight while this round is used
    if (active) {
      const R* sR = stage + b * buf_elems;
      const R* sI = sR + TK * RS;
#pragma unroll 4
      for (int k = q; k < TK; k += KSUB) {
        R xr[4], xi[4], yr[4], yi[4];
        load4(sR + k * RS + 4 * I, xr);
        load4(sI + k * RS + 4 * I, xi);
        load4(sR + k * RS + 4 * J, yr);
        load4(sI + k * RS + 4 * J, yi);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            // conj(x_i) * y_j as four FMAs (the sums' rounding order is the FMAs')
            ar[i][j] = fma(xr[i], yr[j], ar[i][j]);
            ar[i][j] = fma(xi[i], yi[j], ar[i][j]);
            ai[i][j] = fma(xr[i], yi[j], ai[i][j]);
            ai[i][j] = fma(-xi[i], yr[j], ai[i][j]);
          }
      }
      if (kPromote && (r + 1) % kFlushRounds == 0) flush();
    }
    if (r + 1 < nrounds) {
      if (nbuf == 1) __syncthreads();          // one buffer: wait until every thread has used it
      put(nbuf == 2 ? (b ^ 1) : 0, r + 1);     // with two, the other buffer was last read in round r - 1
    }
    __syncthreads();
  }
  if (active || !kPromote) flush();            // FP64: every thread writes its slots (staging is idle)
  __syncthreads();
  if (!active || q != 0) return;
  // combine the KSUB groups in group order, then write the tile
  double* g = gpart + (((int64_t)s * nf + f) * nb) * nb * 2;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int li = 4 * I + i, lj = 4 * J + j;
      if (li >= nb || lj >= nb || lj < li) continue;
      double vr = 0.0, vi = 0.0;
      for (int qq = 0; qq < KSUB; ++qq) {
        vr += acc64[(2 * (4 * i + j)) * kThreads + qq * TPG + (tid % TPG)];
        vi += acc64[(2 * (4 * i + j) + 1) * kThreads + qq * TPG + (tid % TPG)];
      }
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

// Sum of the Grams of nparts spatial slabs (Sec. 3.1: the one reduction of the
// paper's spatial decomposition), [nparts][nf][nb][nb] complex FP64, in part
// order (the same sum, bit for bit, wherever the same parts are given), NaN check.
__global__ void k_gram_sum_parts(const double* __restrict__ parts, int nparts, int nf, int nb,
                                 double* __restrict__ gram, unsigned* __restrict__ flags) {
  const int f = blockIdx.x;
  const int64_t per = (int64_t)nf * nb * nb * 2;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int64_t o = ((int64_t)f * nb * nb + e) * 2;
    double vr = 0.0, vi = 0.0;
    for (int q = 0; q < nparts; ++q) {
      vr += parts[q * per + o];
      vi += parts[q * per + o + 1];
    }
    const int i = e / nb, j = e - i * nb;
    if (i == j && !isfinite(vr)) atomicOr(flags, FLAG_NAN);
    gram[o] = vr;
    gram[o + 1] = vi;
  }
}

// Staging buffers (two when they fit) and shared bytes for element size rb.
int gram_simt_nbuf(int nb, size_t rb, size_t* smem_out) {
  const size_t acc = sizeof(double) * 32 * kThreads;
  const size_t buf = 2 * (size_t)TK * staged_stride(nb) * rb;
  auto total = [&](int n) { return rb == 4 ? acc + n * buf : std::max(acc, n * buf); };
  const int nbuf = total(2) <= kGramSimtSmemMax ? 2 : 1;
  *smem_out = total(nbuf);
  return nbuf;
}

template <typename R>
cudaError_t launch_gram_t(const spod_plan_s& p, int64_t mcount, bool first, cudaStream_t s) {
  const int ntl = (p.nb + 3) / 4;
  const int ntiles = ntl * (ntl + 1) / 2;
  const int groups = (ntiles + TPG - 1) / TPG;
  size_t smem = 0;
  const int nbuf = gram_simt_nbuf(p.nb, sizeof(R), &smem);
  auto kern = k_gram_simt<R>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t per = (mcount + p.gram_splits - 1) / p.gram_splits;
  per = ((per + TK - 1) / TK) * TK;
  dim3 grid((unsigned)p.gram_splits, (unsigned)p.nf, (unsigned)groups);
  kern<<<grid, kThreads, smem, s>>>(static_cast<const R*>(p.d_qhat), p.chunk_points, p.nb, mcount, per,
                                   first ? 1 : 0, nbuf, p.d_gpart, p.nf);
  return cudaGetLastError();
}

}  // namespace

size_t gram_simt_smem_bytes(const spod_plan_s& p) {
  size_t smem = 0;
  gram_simt_nbuf(p.nb, p.f64 ? 8 : 4, &smem);
  return smem;
}

cudaError_t launch_gram_chunk(const spod_plan_s& p, int64_t mcount, bool first, cudaStream_t s) {
  return p.f64 ? launch_gram_t<double>(p, mcount, first, s) : launch_gram_t<float>(p, mcount, first, s);
}

cudaError_t launch_gram_sum_parts(const spod_plan_s& p, const double* parts, int nparts, cudaStream_t s) {
  k_gram_sum_parts<<<p.nf, 256, 0, s>>>(parts, nparts, p.nf, p.nb, p.d_gram, p.d_flags);
  return cudaGetLastError();
}

cudaError_t launch_gram_reduce(const spod_plan_s& p, cudaStream_t s) {
  k_gram_reduce<<<p.nf, 256, 0, s>>>(p.d_gpart, p.gram_splits, p.nf, p.nb, p.kappa, p.d_gram, p.d_flags);
  return cudaGetLastError();
}

}  // namespace spod
