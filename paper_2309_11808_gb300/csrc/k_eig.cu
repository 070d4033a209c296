// Batched Hermitian eigen-decomposition of the nb x nb Grams M_f
// (Eq. spod-discrete-snapshots) and the mode coefficients derived from it.
//
// k_eig_jacobi: one CTA per frequency, FP64 throughout.  Parallel-ordered
// (round-robin) complex Jacobi: in each round nb/2 disjoint plane rotations are
// computed from the current matrix, then applied to all columns (A G, V G) and
// to all rows (G^H A).  Each rotation first makes a_pq real with a diagonal
// phase, then applies the real rotation that annihilates it.  Sweeps stop when
// off(A) <= tol * ||A||_F or at the sweep cap (flagged as not converged).
// Output: eigenvalues descending (ties: lower index first), eigenvectors with
// unit 2-norm and their largest-modulus entry (lowest index on ties) real
// positive.
#include <algorithm>
#include <type_traits>

#include "spod_internal.cuh"

namespace spod {
namespace {

__device__ __forceinline__ double2 cm(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmconj(double2 a, double2 b) {   // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

struct Rot {
  int p, q, act;
  double c, s;
  double2 ph;   // conj(a_pq) / |a_pq|
};

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int i = 0; i < nw; ++i) t += red[i];   // same fixed order in every thread
  return t;
}

__global__ void __launch_bounds__(256) k_eig_jacobi(const double* __restrict__ gram, int n,
                                                    double* __restrict__ lam, double* __restrict__ psi,
                                                    double* __restrict__ gws, unsigned* __restrict__ flags,
                                                    int max_sweeps, double tol) {
  const int f = blockIdx.x;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int np = n + (n & 1);
  const int npairs = np / 2;
  Rot* rot = reinterpret_cast<Rot*>(smem_raw);
  double* red = reinterpret_cast<double*>(rot + npairs);
  double2* A;
  double2* V;
  if (n <= kEigSmemMaxNb) {
    A = reinterpret_cast<double2*>(red + 32);
    V = A + n * n;
  } else {
    A = reinterpret_cast<double2*>(gws) + (size_t)f * 2 * n * n;
    V = A + (size_t)n * n;
  }
  const double2* G = reinterpret_cast<const double2*>(gram) + (size_t)f * n * n;
  const int tid = threadIdx.x, nth = blockDim.x;

  double fro = 0.0;
  for (int e = tid; e < n * n; e += nth) {
    const double2 a = G[e];
    A[e] = a;
    const int i = e / n, j = e - i * n;
    V[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    fro += a.x * a.x + a.y * a.y;
  }
  fro = block_sum(fro, red);
  __syncthreads();

  bool conv = false;
  for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
    double off = 0.0;
    for (int e = tid; e < n * n; e += nth) {
      const int i = e / n, j = e - i * n;
      if (i != j) { const double2 a = A[e]; off += a.x * a.x + a.y * a.y; }
    }
    off = block_sum(off, red);
    if (off <= tol * tol * fro) { conv = true; break; }
    if (sweep == max_sweeps) break;
    for (int r = 0; r < np - 1; ++r) {
      for (int k = tid; k < npairs; k += nth) {
        int a, b;
        if (k == 0) { a = np - 1; b = r; }
        else { a = (r + k) % (np - 1); b = (r - k + np - 1) % (np - 1); }
        Rot R;
        R.p = min(a, b); R.q = max(a, b);
        R.act = 0; R.c = 1.0; R.s = 0.0; R.ph = make_double2(1.0, 0.0);
        if (R.q < n) {
          const double2 apq = A[R.p * n + R.q];
          const double app = A[R.p * n + R.p].x, aqq = A[R.q * n + R.q].x;
          const double mag = hypot(apq.x, apq.y);
          if (mag > 1e-290 && mag > 0x1p-60 * (fabs(app) + fabs(aqq))) {
            R.act = 1;
            R.ph = make_double2(apq.x / mag, -apq.y / mag);
            const double zeta = (aqq - app) / (2.0 * mag);
            const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            R.c = 1.0 / sqrt(1.0 + t * t);
            R.s = t * R.c;
          }
        }
        rot[k] = R;
      }
      __syncthreads();
      // columns: A <- A G, V <- V G with G = diag(1, ph) [[c, s], [-s, c]]
      for (int idx = tid; idx < n * npairs; idx += nth) {
        const int k = idx / n, i = idx - k * n;
        const Rot R = rot[k];
        if (!R.act) continue;
        const double2 g10 = make_double2(-R.s * R.ph.x, -R.s * R.ph.y);
        const double2 g11 = make_double2(R.c * R.ph.x, R.c * R.ph.y);
        double2 cp = A[i * n + R.p], cq = A[i * n + R.q];
        double2 t0 = cm(cq, g10), t1 = cm(cq, g11);
        A[i * n + R.p] = make_double2(cp.x * R.c + t0.x, cp.y * R.c + t0.y);
        A[i * n + R.q] = make_double2(cp.x * R.s + t1.x, cp.y * R.s + t1.y);
        cp = V[i * n + R.p]; cq = V[i * n + R.q];
        t0 = cm(cq, g10); t1 = cm(cq, g11);
        V[i * n + R.p] = make_double2(cp.x * R.c + t0.x, cp.y * R.c + t0.y);
        V[i * n + R.q] = make_double2(cp.x * R.s + t1.x, cp.y * R.s + t1.y);
      }
      __syncthreads();
      // rows: A <- G^H A
      for (int idx = tid; idx < n * npairs; idx += nth) {
        const int k = idx / n, j = idx - k * n;
        const Rot R = rot[k];
        if (!R.act) continue;
        const double2 g10 = make_double2(-R.s * R.ph.x, -R.s * R.ph.y);
        const double2 g11 = make_double2(R.c * R.ph.x, R.c * R.ph.y);
        const double2 rp = A[R.p * n + j], rq = A[R.q * n + j];
        const double2 u = cmconj(g10, rq), v = cmconj(g11, rq);
        A[R.p * n + j] = make_double2(R.c * rp.x + u.x, R.c * rp.y + u.y);
        A[R.q * n + j] = make_double2(R.s * rp.x + v.x, R.s * rp.y + v.y);
      }
      __syncthreads();
      for (int k = tid; k < npairs; k += nth) {
        const Rot R = rot[k];
        if (!R.act) continue;
        A[R.p * n + R.q] = make_double2(0.0, 0.0);
        A[R.q * n + R.p] = make_double2(0.0, 0.0);
        A[R.p * n + R.p].y = 0.0;
        A[R.q * n + R.q].y = 0.0;
      }
      __syncthreads();
    }
  }
  if (!conv && tid == 0) atomicOr(flags, FLAG_NOTCONV);

  // sort descending (stable), normalise, fix phase, scatter
  for (int i = tid; i < n; i += nth) {
    const double li = A[i * n + i].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = A[j * n + j].x;
      rank += (lj > li) || (lj == li && j < i);
    }
    double nrm = 0.0, best = -1.0;
    int piv = 0;
    for (int j = 0; j < n; ++j) {
      const double2 v = V[j * n + i];
      const double m2 = v.x * v.x + v.y * v.y;
      nrm += m2;
      if (m2 > best) { best = m2; piv = j; }
    }
    const double2 pv = V[piv * n + i];
    const double pm = hypot(pv.x, pv.y);
    const double inv = 1.0 / sqrt(nrm);
    const double2 ph = make_double2(pv.x / pm * inv, -pv.y / pm * inv);
    lam[(size_t)f * n + rank] = li;
    double2* out = reinterpret_cast<double2*>(psi) + (size_t)f * n * n;
    for (int j = 0; j < n; ++j) {
      double2 v = cm(V[j * n + i], ph);
      if (j == piv) v.y = 0.0;
      out[j * n + rank] = v;
    }
  }
}

// B_f[l][k] = psi_f[l][k] / sqrt(lambda_k / kappa), zero for lambda_k <= 1e-12 lambda_1.
template <typename R>
__global__ void k_mode_coeffs(const double* __restrict__ lam, const double* __restrict__ psi, int nb,
                              int nmodes, double kappa, R* __restrict__ bmat) {
  const int f = blockIdx.x;
  const double l1 = lam[(size_t)f * nb];
  for (int e = threadIdx.x; e < nb * nmodes; e += blockDim.x) {
    const int l = e / nmodes, k = e - l * nmodes;
    const double lk = lam[(size_t)f * nb + k];
    double sc = 0.0;
    if (lk > 0.0 && lk > 1e-12 * l1) sc = 1.0 / sqrt(lk / kappa);
    const double* src = psi + (((size_t)f * nb + l) * nb + k) * 2;
    R* dst = bmat + (((size_t)f * nb + l) * nmodes + k) * 2;
    dst[0] = (R)(src[0] * sc);
    dst[1] = (R)(src[1] * sc);
  }
}

// Phi[f][k][m] = (1/sqrt(W_m)) sum_l Qhat'[f][l][m] B_f[l][k]   (SIMT)
// One CTA per (tile of 2 * blockDim.x points, frequency).  B_f (all modes,
// rows padded with zeros to a multiple of KG) sits in shared memory; each
// thread takes two adjacent points and walks the modes in groups of KG,
// reading its two points' Qhat pairs from global memory (L1-resident after
// the first group) and B_f as 16-byte broadcast loads.
template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

template <typename R, int KG>
__global__ void __launch_bounds__(128) k_modes_simt(const R* __restrict__ qhat, int64_t rs, int nb, int nmodes,
                                                    int nmp, int64_t mcount, int64_t m0, int64_t M,
                                                    const R* __restrict__ bmat, const R* __restrict__ scale,
                                                    R* __restrict__ phi, int f0, int64_t phioff, int64_t qoff) {
  using V2 = typename Cplx<R>::T;
  const int f = f0 + blockIdx.y;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V2* sB = reinterpret_cast<V2*>(smem_raw);                       // [nb][nmp]
  const V2* Bf = reinterpret_cast<const V2*>(bmat) + (size_t)f * nb * nmodes;
  for (int e = threadIdx.x; e < nb * nmp; e += blockDim.x) {
    const int l = e / nmp, k = e - l * nmp;
    V2 z;
    z.x = 0; z.y = 0;
    sB[e] = k < nmodes ? Bf[l * nmodes + k] : z;
  }
  __syncthreads();
  const int64_t lm = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 2;
  if (lm >= mcount) return;
  const bool two = lm + 1 < mcount;
  const int64_t m = m0 + lm;
  const R s0 = scale[m], s1 = two ? scale[m + 1] : (R)0;
  // point lm + 1 < mpad: the FFT wrote zeros past mcount, so the pair load stays in the chunk
  const R* qf = qhat + (int64_t)f * 2 * nb * rs + qoff + lm;
  const bool vec = (M % 2) == 0;                                  // two points = one aligned 2-complex store
  for (int k0 = 0; k0 < nmodes; k0 += KG) {
    R ar0[KG], ai0[KG], ar1[KG], ai1[KG];
#pragma unroll
    for (int j = 0; j < KG; ++j) { ar0[j] = 0; ai0[j] = 0; ar1[j] = 0; ai1[j] = 0; }
    for (int l = 0; l < nb; ++l) {
      const V2 qr = *reinterpret_cast<const V2*>(qf + (int64_t)l * rs);        // Re, points lm and lm + 1
      const V2 qi = *reinterpret_cast<const V2*>(qf + (int64_t)(nb + l) * rs); // Im
      const V2* bl = sB + l * nmp + k0;
#pragma unroll
      for (int j = 0; j < KG; ++j) {
        const V2 b = bl[j];
        // q * b as FMA chains (four FMAs per complex product and point)
        ar0[j] = fma(qr.x, b.x, ar0[j]);
        ar0[j] = fma(-qi.x, b.y, ar0[j]);
        ai0[j] = fma(qr.x, b.y, ai0[j]);
        ai0[j] = fma(qi.x, b.x, ai0[j]);
        ar1[j] = fma(qr.y, b.x, ar1[j]);
        ar1[j] = fma(-qi.y, b.y, ar1[j]);
        ai1[j] = fma(qr.y, b.y, ai1[j]);
        ai1[j] = fma(qi.y, b.x, ai1[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < KG; ++j) {
      const int k = k0 + j;
      if (k >= nmodes) break;
      R* o = phi + (((int64_t)f * nmodes + k) * M + (m - phioff)) * 2;
      if (two && vec && sizeof(R) == 4) {
        *reinterpret_cast<float4*>(o) = make_float4((float)(ar0[j] * s0), (float)(ai0[j] * s0),
                                                    (float)(ar1[j] * s1), (float)(ai1[j] * s1));
      } else {
        V2 v;
        v.x = ar0[j] * s0; v.y = ai0[j] * s0;
        *reinterpret_cast<V2*>(o) = v;
        if (two) {
          v.x = ar1[j] * s1; v.y = ai1[j] * s1;
          *reinterpret_cast<V2*>(o + 2) = v;
        }
      }
    }
  }
}

}  // namespace

size_t eig_smem_bytes(int nb) {
  const int np = nb + (nb & 1);
  size_t b = sizeof(Rot) * (np / 2) + 32 * sizeof(double);
  b = (b + 15) & ~size_t(15);
  if (nb <= kEigSmemMaxNb) b += 2 * sizeof(double2) * (size_t)nb * nb;
  return b;
}

cudaError_t launch_eig(const spod_plan_s& p, cudaStream_t s) {
  const size_t smem = eig_smem_bytes(p.nb);
  cudaError_t e = cudaFuncSetAttribute(k_eig_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_eig_jacobi<<<p.nf, 256, smem, s>>>(p.d_gram, p.nb, p.d_lam, p.d_psi, p.d_eigws, p.d_flags, 50, 1e-14);
  return cudaGetLastError();
}

// The same eigen-solver launch on caller-chosen buffers (used by the
// allocation-free entry point, which supplies its scratch from a static array).
cudaError_t launch_eig_buffers(const double* gram, int nf, int nb, double* lam, double* psi, double* gws,
                               unsigned* flags, cudaStream_t s) {
  const size_t smem = eig_smem_bytes(nb);
  cudaError_t e = cudaFuncSetAttribute(k_eig_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_eig_jacobi<<<nf, 256, smem, s>>>(gram, nb, lam, psi, gws, flags, 50, 1e-14);
  return cudaGetLastError();
}

cudaError_t launch_mode_coeffs(const spod_plan_s& p, int nmodes, cudaStream_t s) {
  if (p.f64)
    k_mode_coeffs<double><<<p.nf, 256, 0, s>>>(p.d_lam, p.d_psi, p.nb, nmodes, p.kappa,
                                               static_cast<double*>(p.d_bmat));
  else
    k_mode_coeffs<float><<<p.nf, 256, 0, s>>>(p.d_lam, p.d_psi, p.nb, nmodes, p.kappa,
                                              static_cast<float*>(p.d_bmat));
  return cudaGetLastError();
}

#ifndef SPOD_MODES_KGMAX
#define SPOD_MODES_KGMAX 16
#endif
// Modes per group of the FP32 kernel: the fewest groups of at most
// SPOD_MODES_KGMAX modes, split evenly (38 modes: 13 + 13 + 12 instead of
// 16 + 16 + 6 with six idle slots of the last group's FMAs per point).
template <typename R, int KG>
static cudaError_t modes_kernel(void (**kern)(const R*, int64_t, int, int, int, int64_t, int64_t, int64_t, const R*,
                                              const R*, R*, int, int64_t, int64_t)) {
  *kern = k_modes_simt<R, KG>;
  return cudaSuccess;
}

template <typename R>
static cudaError_t launch_modes_t(const spod_plan_s& p, int64_t m0, int64_t mcount, int nmodes, void* d_Phi,
                                  cudaStream_t s, int* nlaunch, bool adjoint, int f0, int f1, int64_t qoff,
                                  int64_t out_ld, int64_t out_off) {
  void (*kern)(const R*, int64_t, int, int, int, int64_t, int64_t, int64_t, const R*, const R*, R*, int, int64_t,
               int64_t) = nullptr;
  int KG = 8;
  if constexpr (sizeof(R) == 8) {
    modes_kernel<R, 8>(&kern);
  } else {
    const int groups = (nmodes + SPOD_MODES_KGMAX - 1) / SPOD_MODES_KGMAX;
    const int need = (nmodes + groups - 1) / groups;
    constexpr int kChoices[] = {4, 8, 10, 13, 16, 20};
    KG = SPOD_MODES_KGMAX;
    for (int c : kChoices)
      if (c >= need && c <= SPOD_MODES_KGMAX) { KG = c; break; }
    switch (KG) {
      case 4: modes_kernel<R, 4>(&kern); break;
      case 8: modes_kernel<R, 8>(&kern); break;
      case 10: modes_kernel<R, 10>(&kern); break;
      case 13: modes_kernel<R, 13>(&kern); break;
      case 16: modes_kernel<R, 16>(&kern); break;
      default: modes_kernel<R, SPOD_MODES_KGMAX>(&kern); KG = SPOD_MODES_KGMAX; break;
    }
  }
  const int nmp = (nmodes + KG - 1) / KG * KG;
  const size_t smem = sizeof(typename Cplx<R>::T) * (size_t)p.nb * nmp;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  constexpr int threads = 128;
  dim3 grid((unsigned)((mcount + 2 * threads - 1) / (2 * threads)), (unsigned)(f1 - f0));
  const int64_t ld = out_ld ? out_ld : (p.phi_ld && !adjoint) ? p.phi_ld : p.M;
  kern<<<grid, threads, smem, s>>>(static_cast<const R*>(p.d_qhat), p.chunk_points, p.nb, nmodes, nmp, mcount, m0,
                                   ld, static_cast<const R*>(p.d_bmat),
                                   static_cast<const R*>(adjoint ? p.d_sqrtW : p.d_rsqrtW), static_cast<R*>(d_Phi),
                                   f0, out_ld ? out_off : adjoint ? 0 : p.phi_off, qoff);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ++*nlaunch;
  return cudaSuccess;
}

cudaError_t launch_modes_chunk(const spod_plan_s& p, int64_t m0, int64_t mcount, int nmodes, void* d_Phi,
                               cudaStream_t s, int* nlaunch, bool adjoint, int f0, int f1, int64_t qoff,
                               int64_t out_ld, int64_t out_off) {
  if (f1 < 0) f1 = p.nf;
  if (f0 < 0 || f1 > p.nf || f0 >= f1 || qoff % 2 != 0) return cudaErrorInvalidValue;
  return p.f64 ? launch_modes_t<double>(p, m0, mcount, nmodes, d_Phi, s, nlaunch, adjoint, f0, f1, qoff, out_ld,
                                        out_off)
               : launch_modes_t<float>(p, m0, mcount, nmodes, d_Phi, s, nlaunch, adjoint, f0, f1, qoff, out_ld,
                                       out_off);
}

}  // namespace spod
