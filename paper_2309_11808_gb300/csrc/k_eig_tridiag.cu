// Batched Hermitian eigen-decomposition of the Grams M_f by Householder
// tridiagonalisation and implicit QL iteration (FP64, one CTA per frequency).
//
// 1. Reduction (n-1 steps): for column k, the reflector H_k = I - tau v v^H
//    (v[0] = 1) with H_k^H (a, x)^T = (beta, 0)^T, beta real, annihilates
//    A[k+2:, k] and makes the subdiagonal real; the trailing block is updated
//    as A <- H_k^H A H_k = A - v w^H - w v^H with p = tau A v and
//    w = p - (tau/2)(p^H v) v.  Then A = Q T Q^H, Q = H_0 H_1 ... H_{n-2}, T real
//    symmetric tridiagonal.
// 2. Implicit QL with Wilkinson shifts on (d, e): thread 0 runs each sweep's
//    chain of plane rotations and records them; all threads then apply the
//    sequence to their rows of the real eigenvector matrix Z.
// 3. Back-transform V = Q Z, columns in parallel.
// 4. Eigenvalues descending (ties: lower index first); eigenvectors unit
//    2-norm with the largest-modulus entry (lowest index on ties) real positive.
// About 10 n^3 FP64 operations against ~150 n^3 for the cyclic Jacobi solver.
#include "spod_internal.cuh"

namespace spod {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxIter = 60;           // QL iterations per eigenvalue

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {   // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__device__ double2 block_sum2(double2 v, double2* red) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double2 t = make_double2(0.0, 0.0);
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { t.x += red[i].x; t.y += red[i].y; }
  return t;
}

__global__ void __launch_bounds__(kThreads) k_eig_tridiag(const double* __restrict__ gram, int n,
                                                          double* __restrict__ lam, double* __restrict__ psi,
                                                          double* __restrict__ gws, unsigned* __restrict__ flags) {
  const int f = blockIdx.x;
  const int tid = threadIdx.x, nth = blockDim.x;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* red = reinterpret_cast<double2*>(smem_raw);          // [32]
  double2* tau = red + 32;                                       // [n]
  double2* pv = tau + n;                                         // [n] p / w
  double* d = reinterpret_cast<double*>(pv + n);                 // [n]
  double* e = d + n;                                             // [n]
  double* rc = e + n;                                            // [n] rotation cosines
  double* rsn = rc + n;                                          // [n] rotation sines
  int* ctl = reinterpret_cast<int*>(rsn + n);                    // [4] control words
  // per frequency: A [n][n] complex, Lv [n][n] complex (reflector copy), Z [n][n] real
  double2* A;
  {
    uint8_t* after = reinterpret_cast<uint8_t*>(ctl + 4);
    after = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(after) + 15) & ~uintptr_t(15));
    // per-frequency stride rounded up to an even number of doubles: double2 needs 16-byte alignment
    const size_t stride = ((size_t)5 * n * n + 1) & ~(size_t)1;
    A = (n <= kEigSmemMaxNb) ? reinterpret_cast<double2*>(after) : reinterpret_cast<double2*>(gws + (size_t)f * stride);
  }
  double2* Lv = A + (size_t)n * n;
  double* Z = reinterpret_cast<double*>(Lv + (size_t)n * n);
  double2* V = A;   // the back-transform overwrites A once the reflectors are copied to Lv
  const double2* G = reinterpret_cast<const double2*>(gram) + (size_t)f * n * n;
  for (int i = tid; i < n * n; i += nth) A[i] = G[i];
  __syncthreads();

  // ---------------- 1. Householder reduction to real tridiagonal form
  for (int k = 0; k + 1 < n; ++k) {
    const int m = n - k - 1;                    // length of x = A[k+1:, k]
    double2 part = make_double2(0.0, 0.0);
    for (int i = 1 + tid; i < m; i += nth) {
      const double2 x = A[(k + 1 + i) * n + k];
      part.x += x.x * x.x + x.y * x.y;
    }
    const double xn2 = block_sum2(part, red).x;   // |x[1:]|^2
    if (tid == 0) {
      const double2 alpha = A[(k + 1) * n + k];
      double2 t = make_double2(0.0, 0.0);
      double beta = alpha.x;                     // stays alpha when no reflection is needed
      double2 scale = make_double2(0.0, 0.0);
      if (xn2 > 0.0 || alpha.y != 0.0) {
        const double nrm = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2);
        beta = alpha.x >= 0.0 ? -nrm : nrm;
        t = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
        // scale = 1 / (alpha - beta)
        const double2 den = make_double2(alpha.x - beta, alpha.y);
        const double dd = den.x * den.x + den.y * den.y;
        scale = make_double2(den.x / dd, -den.y / dd);
      }
      tau[k] = t;
      e[k] = beta;
      pv[0] = scale;                             // broadcast
    }
    __syncthreads();
    const double2 t = tau[k];
    const double2 scale = pv[0];
    __syncthreads();
    if (t.x == 0.0 && t.y == 0.0) continue;
    // v = (1, x[1:] * scale), stored in place below the subdiagonal
    for (int i = 1 + tid; i < m; i += nth) A[(k + 1 + i) * n + k] = cmul(A[(k + 1 + i) * n + k], scale);
    if (tid == 0) A[(k + 1) * n + k] = make_double2(1.0, 0.0);
    __syncthreads();
    // p = tau * A22 v   (A22 = A[k+1:, k+1:])
    for (int i = tid; i < m; i += nth) {
      double2 s = make_double2(0.0, 0.0);
      const double2* row = A + (size_t)(k + 1 + i) * n + (k + 1);
      for (int j = 0; j < m; ++j) {
        const double2 a = row[j], v = A[(k + 1 + j) * n + k];
        s.x += a.x * v.x - a.y * v.y;
        s.y += a.x * v.y + a.y * v.x;
      }
      pv[i] = cmul(t, s);
    }
    __syncthreads();
    // w = p - (tau/2) (p^H v) v
    double2 dot = make_double2(0.0, 0.0);
    for (int i = tid; i < m; i += nth) {
      const double2 c = cmulc(pv[i], A[(k + 1 + i) * n + k]);
      dot.x += c.x; dot.y += c.y;
    }
    dot = block_sum2(dot, red);
    const double2 al = cmul(make_double2(-0.5 * t.x, -0.5 * t.y), dot);
    __syncthreads();
    for (int i = tid; i < m; i += nth) {
      const double2 v = A[(k + 1 + i) * n + k];
      const double2 c = cmul(al, v);
      pv[i] = make_double2(pv[i].x + c.x, pv[i].y + c.y);
    }
    __syncthreads();
    // A22 -= v w^H + w v^H
    for (int idx = tid; idx < m * m; idx += nth) {
      const int i = idx / m, j = idx - i * m;
      const double2 vi = A[(k + 1 + i) * n + k], vj = A[(k + 1 + j) * n + k];
      const double2 wi = pv[i], wj = pv[j];
      double2& a = A[(k + 1 + i) * n + (k + 1 + j)];
      // v_i conj(w_j) + w_i conj(v_j)
      a.x -= (vi.x * wj.x + vi.y * wj.y) + (wi.x * vj.x + wi.y * vj.y);
      a.y -= (vi.y * wj.x - vi.x * wj.y) + (wi.y * vj.x - wi.x * vj.y);
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += nth) d[i] = A[i * n + i].x;
  for (int idx = tid; idx < n * n; idx += nth) Z[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
  if (tid == 0) {
    e[n - 1] = 0.0;
    ctl[0] = 0;   // not-converged flag
  }
  __syncthreads();

  // ---------------- 2. implicit QL with Wilkinson shifts; e[i] couples d[i], d[i+1]
  // Warp 0 finds the end mm of the unreduced block (lanes test 32 indices at
  // once), lane 0 runs the rotation chain.  FP64 is slow on this part, so the
  // chain forms each rotation from one reciprocal square root (r^2 = f^2 + g^2,
  // s = f / r, c = g / r) instead of hypot and two divisions; the scaled hypot
  // path is kept for r^2 outside [2^-960, 2^960].
  // A coupling also counts as negligible below eps * ||T||_inf: dropping it moves
  // no eigenvalue by more than that (Weyl), the normwise accuracy of the
  // reduction itself.  Without this floor the purely relative test can stall on
  // a cluster of rounding-level eigenvalues of a rank-deficient Gram (nb > M).
  const int warp = tid >> 5, lane = tid & 31;
  double tfloor = 0.0;
  if (warp == 0) {
    double m = 0.0;
    for (int i = lane; i < n; i += 32) m = fmax(m, fabs(d[i]) + fabs(e[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    tfloor = 0x1p-53 * m;
  }
  for (int l = 0; l < n; ++l) {
    for (int iter = 0;; ++iter) {
      if (warp == 0) {
        int mm = n - 1;
        for (int base = l; base < n - 1; base += 32) {
          const int i = base + lane;
          bool split = false;
          if (i < n - 1) split = fabs(e[i]) <= fmax(0x1p-53 * (fabs(d[i]) + fabs(d[i + 1])), tfloor);
          const unsigned bal = __ballot_sync(0xffffffffu, split);
          if (bal) { mm = base + __ffs(bal) - 1; break; }
        }
        if (lane == 0) {
          int nrot = 0;
          if (mm != l) {
            if (iter >= kMaxIter) {
              ctl[0] = 1;
              mm = l;                                    // give up on this eigenvalue
            } else {
              double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
              double r = sqrt(fma(g, g, 1.0));
              g = d[mm] - d[l] + e[l] / (g + (g >= 0.0 ? r : -r));
              double s = 1.0, c = 1.0, p = 0.0;
              bool underflow = false;
              for (int i = mm - 1; i >= l; --i) {
                const double ff = s * e[i];
                const double b = c * e[i];
                const double r2 = fma(ff, ff, g * g);
                if (r2 > 0x1p-960 && r2 < 0x1p960) {
                  const double ri = rsqrt(r2);
                  r = r2 * ri;
                  s = ff * ri;
                  c = g * ri;
                } else {
                  r = hypot(ff, g);
                  if (r == 0.0) {
                    e[i + 1] = 0.0;
                    d[i + 1] -= p;
                    e[mm] = 0.0;
                    underflow = true;
                    break;
                  }
                  s = ff / r;
                  c = g / r;
                }
                e[i + 1] = r;
                g = d[i + 1] - p;
                r = fma(d[i] - g, s, 2.0 * c * b);
                p = s * r;
                d[i + 1] = g + p;
                g = fma(c, r, -b);
                rc[nrot] = c;
                rsn[nrot] = s;
                ++nrot;
              }
              if (!underflow) {
                d[l] -= p;
                e[l] = g;
                e[mm] = 0.0;
              }
            }
          }
          ctl[1] = mm;
          ctl[2] = nrot;
        }
      }
      __syncthreads();
      const int mm = ctl[1], nrot = ctl[2];
      // apply the recorded rotations (columns i+1, i for i = mm-1 down) to every row of Z
      for (int row = tid; row < n; row += nth) {
        double* zr = Z + (size_t)row * n;
        for (int q = 0; q < nrot; ++q) {
          const int i = mm - 1 - q;
          const double c = rc[q], s = rsn[q];
          const double fz = zr[i + 1];
          zr[i + 1] = fma(s, zr[i], c * fz);
          zr[i] = fma(c, zr[i], -s * fz);
        }
      }
      __syncthreads();
      if (mm == l) break;
    }
  }
  if (tid == 0 && ctl[0]) atomicOr(flags, FLAG_NOTCONV);

  // ---------------- 3. V = Q Z: apply H_{n-2}, ..., H_0 to Z
  double2* vs = pv;   // s_j of one reflector
  for (int idx = tid; idx < n * n; idx += nth) {
    const int i = idx / n, k = idx - i * n;
    Lv[idx] = (i > k) ? A[idx] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += nth) V[idx] = make_double2(Z[idx], 0.0);
  __syncthreads();
  for (int k = n - 2; k >= 0; --k) {
    const double2 t = tau[k];
    if (t.x == 0.0 && t.y == 0.0) continue;
    const int m = n - k - 1;
    // s_j = v^H V[k+1:, j] ; V[k+1:, j] -= tau v s_j
    for (int j = tid; j < n; j += nth) {
      double2 s = make_double2(0.0, 0.0);
      for (int i = 0; i < m; ++i) {
        const double2 c = cmulc(Lv[(k + 1 + i) * n + k], V[(k + 1 + i) * n + j]);
        s.x += c.x; s.y += c.y;
      }
      vs[j] = cmul(t, s);
    }
    __syncthreads();
    for (int idx = tid; idx < m * n; idx += nth) {
      const int i = idx / n, j = idx - i * n;
      const double2 c = cmul(Lv[(k + 1 + i) * n + k], vs[j]);
      double2& vv = V[(k + 1 + i) * n + j];
      vv.x -= c.x;
      vv.y -= c.y;
    }
    __syncthreads();
  }

  // ---------------- 4. sort, normalise, phase, scatter
  for (int i = tid; i < n; i += nth) {
    const double li = d[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = d[j];
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
    const double2 pvv = V[piv * n + i];
    const double pm = hypot(pvv.x, pvv.y);
    const double inv = 1.0 / sqrt(nrm);
    const double2 ph = make_double2(pvv.x / pm * inv, -pvv.y / pm * inv);
    lam[(size_t)f * n + rank] = li;
    double2* out = reinterpret_cast<double2*>(psi) + (size_t)f * n * n;
    for (int j = 0; j < n; ++j) {
      double2 v = cmul(V[j * n + i], ph);
      if (j == piv) v.y = 0.0;
      out[j * n + rank] = v;
    }
  }
}

}  // namespace

size_t eig_tridiag_smem_bytes(int nb) {
  size_t b = sizeof(double2) * (32 + 2 * (size_t)nb) + sizeof(double) * 4 * (size_t)nb + 4 * sizeof(int) + 16;
  if (nb <= kEigSmemMaxNb) b += sizeof(double) * 5 * (size_t)nb * nb;
  return b;
}

size_t eig_tridiag_gws_doubles(int nb, int nf) {
  // per frequency: A (n^2 complex) + reflector copy (n^2 complex) + Z (n^2 real)
  return (size_t)nf * (((size_t)5 * nb * nb + 1) & ~(size_t)1);
}

cudaError_t launch_eig_tridiag(const spod_plan_s& p, cudaStream_t s) {
  const size_t smem = eig_tridiag_smem_bytes(p.nb);
  cudaError_t e = cudaFuncSetAttribute(k_eig_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_eig_tridiag<<<p.nf, kThreads, smem, s>>>(p.d_gram, p.nb, p.d_lam, p.d_psi, p.d_eigws, p.d_flags);
  return cudaGetLastError();
}

}  // namespace spod
