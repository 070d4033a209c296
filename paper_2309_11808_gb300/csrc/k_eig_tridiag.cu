// Batched Hermitian eigen-decomposition of the Grams M_f by Householder
// tridiagonalisation and implicit QL iteration (one 256-thread CTA per
// frequency).
//
// 1. Reduction (n-1 steps): for column k, the reflector H_k = I - tau v v^H
//    (v[0] = 1) with H_k^H (a, x)^T = (beta, 0)^T, beta real, annihilates
//    A[k+2:, k] and makes the subdiagonal real; the trailing block is updated
//    as A <- H_k^H A H_k = A - v w^H - w v^H with p = tau A v and
//    w = p - (tau/2)(p^H v) v.  Then A = Q T Q^H, Q = H_0 H_1 ... H_{n-2}, T real
//    symmetric tridiagonal.
// 2. Three warp roles run at once:
//    * warp 0: implicit QL with Wilkinson shifts on (d, e); lane 0 runs each
//      sweep's chain of plane rotations and publishes (cosine, sine) into one
//      of two buffers;
//    * warps 1-2: apply each published sweep to the rows of the real
//      eigenvector matrix Z, one buffer behind the chain;
//    * warps 3-7: form Q explicitly from the stored reflectors (FP64).
//    Named barriers hand the two rotation buffers back and forth.
// 3. V = Q Z (FP64, all threads).
// 4. Eigenvalues descending (ties: lower index first); eigenvectors unit
//    2-norm with the largest-modulus entry (lowest index on ties) real positive.
//
// On this part a dependent FP64 operation costs about 14 times a FP32 one, and
// every FP64 warp instruction occupies the FP64 pipe about as long whatever
// the number of active lanes.  So steps 1 and 2 run in FP64 only for the FP64
// precision; for the others the reduction (on A scaled by a power of two),
// the one-thread rotation chain (on T scaled by a power of two) and the Z
// rotations run in double-FP32 (an unevaluated sum of two floats, about 48
// bits), and Q, V = Q Z and step 4 in FP64.  Matrices keep odd row strides (in 8-
// and 16-byte units) so column walks fall in distinct shared-memory banks, and
// the reduction's matrix-vector product reads columns (A is Hermitian) split
// over all warps.
#include "spod_internal.cuh"

namespace spod {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxIter = 60;           // QL iterations per eigenvalue (default; the plan may set another cap)
constexpr int kBarFull = 1;            // named barriers 1, 2: rotation buffer published
constexpr int kBarEmpty = 3;           // named barriers 3, 4: rotation buffer applied
constexpr int kBarQ = 5;               // named barrier of the Q-forming warps
constexpr int kRotThreads = 96;        // warp 0 + warps 1-2
constexpr int kQThreads = kThreads - kRotThreads;

__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

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

__host__ __device__ constexpr int odd_stride(int n) { return n | 1; }

// ---- double-FP32 ("df64") arithmetic: value = h + l, |l| <= ulp(h) / 2.
// Error-free transformations (Knuth's TwoSum, Dekker's Fast2Sum, the FMA
// product) and the double-word sum and product of Joldes, Muller and Popescu
// (ACM TOMS 44(2), 2017: accurate DW + DW, DW x DW).  Explicit _rn intrinsics
// keep the compiler from contracting or reordering them.
struct dw {
  float h, l;
};
__device__ __forceinline__ dw dw_of(float a) { return {a, 0.0f}; }
__device__ __forceinline__ dw two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float t = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, t)), __fsub_rn(b, t));
  return {s, e};
}
__device__ __forceinline__ dw fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dw dw_add(dw x, dw y) {
  const dw s = two_sum(x.h, y.h), t = two_sum(x.l, y.l);
  const dw v = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
  return fast_two_sum(v.h, __fadd_rn(t.l, v.l));
}
__device__ __forceinline__ dw dw_neg(dw x) { return {-x.h, -x.l}; }
__device__ __forceinline__ dw dw_sub(dw x, dw y) { return dw_add(x, dw_neg(y)); }
__device__ __forceinline__ dw dw_mul(dw x, dw y) {
  const float ch = __fmul_rn(x.h, y.h);
  const float cl1 = __fmaf_rn(x.h, y.h, -ch);
  const float tl1 = __fmaf_rn(x.h, y.l, __fmul_rn(x.l, y.l));
  const float cl2 = __fmaf_rn(x.l, y.h, tl1);
  return fast_two_sum(ch, __fadd_rn(cl1, cl2));
}
__device__ __forceinline__ dw dw_mul2(dw x) { return {2.0f * x.h, 2.0f * x.l}; }   // exact
// x / y: an FP32 quotient and two residual corrections.
__device__ __forceinline__ dw dw_div(dw x, dw y) {
  const float q1 = __fdividef(x.h, y.h);
  const dw r1 = dw_sub(x, dw_mul(y, dw_of(q1)));
  const float q2 = __fdividef(r1.h, y.h);
  const dw r2 = dw_sub(r1, dw_mul(y, dw_of(q2)));
  const float q3 = __fdividef(r2.h, y.h);
  return dw_add(fast_two_sum(q1, q2), dw_of(q3));
}
// Sum of two non-negative df64 values (no cancellation: the short form of
// the double-word sum, whose error bound holds for operands of one sign).
__device__ __forceinline__ dw dw_add_pos(dw x, dw y) {
  const dw s = two_sum(x.h, y.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}
// 1 / sqrt(x), x > 0 normal: y0 = rsqrtf(x_h), then the second-order step
// y = y0 (1 + e/2 + 3 e^2/8) on the residual e = 1 - x y0^2 (|e| ~ 2^-22),
// formed with FMAs: x_h y0 = h + hl exactly, 1 - h y0 and the rest of x y0^2
// folded in by one more FMA (error of e about 2^-45, of y about 2^-46).
__device__ __forceinline__ dw dw_rsqrt(dw x) {
  const float y0 = rsqrtf(x.h);
  const float h = __fmul_rn(x.h, y0);
  const float hl = __fmaf_rn(x.h, y0, -h);
  const float t = __fmaf_rn(x.l, y0, hl);             // x y0 - h
  const float e = __fmaf_rn(-t, y0, __fmaf_rn(-h, y0, 1.0f));
  const float u = __fmul_rn(e, __fmaf_rn(0.375f, e, 0.5f));
  return fast_two_sum(y0, __fmul_rn(y0, u));
}
__device__ __forceinline__ dw dw_from_double(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double dw_to_double(dw v) { return (double)v.h + (double)v.l; }

// One implicit QL sweep with a Wilkinson shift over the unreduced block
// [l, mm] of (d, e) (one thread); records the rotations' cosines and sines for
// the eigenvector update and returns their number.  FP64 form.  The sweep is
// the implicit shifted QL step for symmetric tridiagonal matrices of Bowdler,
// Martin, Reinsch and Wilkinson (the tql2 procedure of the Handbook for
// Automatic Computation, 1968/1971): a Givens chain chasing the bulge from
// the bottom of the block to its top, in its published order of updates.
__device__ __noinline__ int ql_sweep_f64(double* d, double* e, int l, int mm, double* rc, double* rsn) {
  // shift: g = (d_l+1 - d_l) / (2 e_l), r = sqrt(g^2 + 1), g = d_mm - d_l + e_l / (g + sign(g) r)
  double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
  double r = sqrt(fma(g, g, 1.0));
  g = d[mm] - d[l] + e[l] / (g + (g >= 0.0 ? r : -r));
  double s = 1.0, c = 1.0, p = 0.0;
  int nrot = 0;
  for (int i = mm - 1; i >= l; --i) {
    const double ff = s * e[i];
    const double b = c * e[i];
    const double r2 = fma(ff, ff, g * g);
    if (r2 > 0x1p-960 && r2 < 0x1p960) {     // one reciprocal square root
      const double ri = rsqrt(r2);
      r = r2 * ri;
      s = ff * ri;
      c = g * ri;
    } else {                                  // scaled form outside that range
      r = hypot(ff, g);
      if (r == 0.0) {                         // the block splits at i + 1
        e[i + 1] = 0.0;
        d[i + 1] -= p;
        e[mm] = 0.0;
        return nrot;
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
  d[l] -= p;
  e[l] = g;
  e[mm] = 0.0;
  return nrot;
}

// The same sweep in df64 on the scaled (d, e) held as (h, l) float pairs.
__device__ __noinline__ int ql_sweep_dw(float2* dd, float2* ee, int l, int mm, double* rc, double* rsn) {
  auto D = [&](int i) { const float2 v = dd[i]; return dw{v.x, v.y}; };
  auto E = [&](int i) { const float2 v = ee[i]; return dw{v.x, v.y}; };
  auto setD = [&](int i, dw v) { dd[i] = make_float2(v.h, v.l); };
  auto setE = [&](int i, dw v) { ee[i] = make_float2(v.h, v.l); };
  const dw dl = D(l), el = E(l);
  dw g = dw_div(dw_sub(D(l + 1), dl), dw_mul2(el));
  const dw t = dw_add(dw_mul(g, g), dw_of(1.0f));
  const dw r0 = dw_mul(t, dw_rsqrt(t));
  g = dw_add(dw_sub(D(mm), dl), dw_div(el, g.h >= 0.0f ? dw_add(g, r0) : dw_sub(g, r0)));
  dw s = dw_of(1.0f), c = dw_of(1.0f), p = dw_of(0.0f);
  int nrot = 0;
  // d[i+1], d[i] and e[i] of the rotation at i, loaded one rotation ahead
  // (the rotation at i writes only d[i+1] and e[i+1]), so the chain does
  // not wait on shared-memory loads
  dw dn = D(mm), di = D(mm - 1), ei = E(mm - 1);
  for (int i = mm - 1; i >= l; --i) {
    const int inext = i > l ? i - 1 : i;
    const dw di_next = D(inext), ei_next = E(inext);
    dw ff = dw_mul(s, ei), gg = g;
    const dw b = dw_mul(c, ei);
    float post = 1.0f;
    dw r2 = dw_add_pos(dw_mul(ff, ff), dw_mul(gg, gg));
    if (r2.h < 0x1p-100f) {                 // tiny pair: rescale by an exact power of two
      ff = {ff.h * 0x1p64f, ff.l * 0x1p64f};
      gg = {gg.h * 0x1p64f, gg.l * 0x1p64f};
      post = 0x1p-64f;
      r2 = dw_add_pos(dw_mul(ff, ff), dw_mul(gg, gg));
    }
    if (!(r2.h > 0x1p-120f)) {              // both negligible: the block splits at i + 1
      setE(i + 1, dw_of(0.0f));
      setD(i + 1, dw_sub(dn, p));
      setE(mm, dw_of(0.0f));
      return nrot;
    }
    const dw ri = dw_rsqrt(r2);
    const dw rr = dw_mul(r2, ri);
    setE(i + 1, {rr.h * post, rr.l * post});
    s = dw_mul(ff, ri);
    c = dw_mul(gg, ri);
    g = dw_sub(dn, p);
    const dw u = dw_add(dw_mul(dw_sub(di, g), s), dw_mul2(dw_mul(c, b)));
    p = dw_mul(s, u);
    setD(i + 1, dw_add(g, p));
    g = dw_sub(dw_mul(c, u), b);
    // handed to the appliers as (h, l) pairs: no FP64 operation in the chain
    reinterpret_cast<float2*>(rc)[nrot] = make_float2(c.h, c.l);
    reinterpret_cast<float2*>(rsn)[nrot] = make_float2(s.h, s.l);
    ++nrot;
    dn = di;
    di = di_next;
    ei = ei_next;
  }
  setD(l, dw_sub(D(l), p));
  setE(l, g);
  setE(mm, dw_of(0.0f));
  return nrot;
}

// Warp 0: QL on (d, e), publishing every sweep with rotations into buffer
// (published count) & 1; then a terminator (nrot = -1).  Before a buffer is
// rewritten the appliers must have released it; at the end the last buffer
// is waited for, so every arrival on the named barriers is matched.
template <bool kDW>
__device__ void ql_producer(double* d, double* e, int n, double* rc, double* rsn, int* ctl, int max_iter) {
  const int lane = threadIdx.x & 31;
  double tn = 0.0;
  for (int i = lane; i < n; i += 32) tn = fmax(tn, fabs(d[i]) + fabs(e[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0));
  for (int o = 16; o > 0; o >>= 1) tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
  // A coupling counts as negligible when |e_i| <= u (|d_i| + |d_i+1|) or
  // |e_i| <= u ||T||_inf (u = 2^-53 in FP64, 2^-47 in df64): dropping it moves
  // no eigenvalue by more than that (Weyl).  Without the absolute floor the
  // relative test can stall on a cluster of rounding-level eigenvalues of a
  // rank-deficient Gram (nb > M).
  double sc = 1.0;
  float2* dd = reinterpret_cast<float2*>(d);
  float2* ee = reinterpret_cast<float2*>(e);
  if constexpr (kDW) {
    sc = scalbn(1.0, tn > 0.0 ? -ilogb(tn) : 0);      // ||T||_inf * sc in [1, 2)
    for (int i = lane; i < n; i += 32) {
      const dw a = dw_from_double(d[i] * sc), b = dw_from_double(e[i] * sc);
      dd[i] = make_float2(a.h, a.l);
      ee[i] = make_float2(b.h, b.l);
    }
    __syncwarp();
  }
  const double tfloor = 0x1p-53 * tn;
  const float tfloor_f = 0x1p-47f * (float)(tn * sc);
  int pub = 0;
  for (int l = 0; l < n; ++l) {
    for (int iter = 0;; ++iter) {
      int mm = n - 1;
      for (int base = l; base < n - 1; base += 32) {
        const int i = base + lane;
        bool split = false;
        if (i < n - 1) {
          if constexpr (kDW)
            split = fabsf(ee[i].x) <= fmaxf(0x1p-47f * (fabsf(dd[i].x) + fabsf(dd[i + 1].x)), tfloor_f);
          else
            split = fabs(e[i]) <= fmax(0x1p-53 * (fabs(d[i]) + fabs(d[i + 1])), tfloor);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, split);
        if (bal) { mm = base + __ffs(bal) - 1; break; }
      }
      if (mm == l) break;
      if (iter >= max_iter) {                 // give up on this eigenvalue
        if (lane == 0) ctl[0] = 1;
        break;
      }
      const int slot = pub & 1;
      if (pub >= 2) named_sync(kBarEmpty + slot, kRotThreads);
      int nrot = 0;
      if (lane == 0) {
        double* rcs = rc + slot * n;
        double* rss = rsn + slot * n;
        if constexpr (kDW) nrot = ql_sweep_dw(dd, ee, l, mm, rcs, rss);
        else nrot = ql_sweep_f64(d, e, l, mm, rcs, rss);
        ctl[2 + 2 * slot] = mm;
        ctl[3 + 2 * slot] = nrot;
      }
      nrot = __shfl_sync(0xffffffffu, nrot, 0);
      __syncwarp();
      if (nrot > 0) {
        __threadfence_block();
        named_arrive(kBarFull + slot, kRotThreads);
        ++pub;
      }
    }
  }
  const int slot = pub & 1;
  if (pub >= 2) named_sync(kBarEmpty + slot, kRotThreads);
  if (lane == 0) ctl[3 + 2 * slot] = -1;
  __syncwarp();
  __threadfence_block();
  named_arrive(kBarFull + slot, kRotThreads);
  if (pub >= 1) named_sync(kBarEmpty + ((pub - 1) & 1), kRotThreads);
  if constexpr (kDW) {
    for (int i = lane; i < n; i += 32) {
      const float2 a = dd[i];
      d[i] = dw_to_double({a.x, a.y}) / sc;
    }
  }
}

// Warps 1-2: apply each published sweep (columns i+1, i for i = mm-1 down) to
// the rows of Z.  The value of column i a rotation leaves is the next
// rotation's column i+1, so it stays in a register.  FP64 form: Z in FP64.
// df64 form (kDW): the rotations arrive as (h, l) float pairs and each row of
// Z is rotated in df64, held as float pairs in Z's storage; FP64 is the
// scarce pipe on this part and the appliers of a CTA would otherwise occupy
// it for every rotation of the chain.  Z returns to FP64 at the end.
template <bool kDW>
__device__ void ql_applier(double* Z, int ldz, int n, const double* rc, const double* rsn, const int* ctl) {
  const int t = threadIdx.x - 32;
  float2* Zf = reinterpret_cast<float2*>(Z);
  if constexpr (kDW) {
    for (int row = t; row < n; row += 64)
      for (int c = 0; c < n; ++c) Zf[(size_t)row * ldz + c] = make_float2((float)Z[(size_t)row * ldz + c], 0.0f);
  }
  for (int q = 0;; ++q) {
    const int slot = q & 1;
    named_sync(kBarFull + slot, kRotThreads);
    const int mm = ctl[2 + 2 * slot], nrot = ctl[3 + 2 * slot];
    if (nrot < 0) break;
    if constexpr (kDW) {
      const float2* rcs = reinterpret_cast<const float2*>(rc) + slot * n;
      const float2* rss = reinterpret_cast<const float2*>(rsn) + slot * n;
      for (int row = t; row < n; row += 64) {
        float2* zr = Zf + (size_t)row * ldz;
        dw fz = {zr[mm].x, zr[mm].y};
        for (int j = 0; j < nrot; ++j) {
          const int i = mm - 1 - j;
          const float2 c2 = rcs[j], s2 = rss[j];
          const dw c = {c2.x, c2.y}, s = {s2.x, s2.y};
          const float2 zi2 = zr[i];
          const dw zi = {zi2.x, zi2.y};
          const dw up = dw_add(dw_mul(s, zi), dw_mul(c, fz));
          zr[i + 1] = make_float2(up.h, up.l);
          fz = dw_sub(dw_mul(c, zi), dw_mul(s, fz));
        }
        if (nrot > 0) zr[mm - nrot] = make_float2(fz.h, fz.l);
      }
    } else {
      const double* rcs = rc + slot * n;
      const double* rss = rsn + slot * n;
      for (int row = t; row < n; row += 64) {
        double* zr = Z + (size_t)row * ldz;
        for (int j = 0; j < nrot; ++j) {
          const int i = mm - 1 - j;
          const double c = rcs[j], s = rss[j];
          const double fz = zr[i + 1];
          zr[i + 1] = fma(s, zr[i], c * fz);
          zr[i] = fma(c, zr[i], -s * fz);
        }
      }
    }
    named_arrive(kBarEmpty + slot, kRotThreads);
  }
  if constexpr (kDW) {
    for (int row = t; row < n; row += 64)
      for (int c = 0; c < n; ++c) {
        const float2 v = Zf[(size_t)row * ldz + c];
        Z[(size_t)row * ldz + c] = (double)v.x + (double)v.y;
      }
  }
}

// Warps 3-7: Q = H_0 H_1 ... H_{n-2} from the reflectors stored below the
// subdiagonal of A (v_0 = 1 in place), applied to I in reverse order; after
// H_{n-2} .. H_{k+1}, rows and columns up to k are still those of I, so H_k
// touches the block [k+1:, k+1:] only.
__device__ void form_q(const double2* A, double2* Qm, int lda, int n, const double2* tau, double2* sv) {
  const int t = threadIdx.x - kRotThreads;
  for (int idx = t; idx < n * n; idx += kQThreads) {
    const int r = idx / n, c = idx - r * n;
    Qm[(size_t)r * lda + c] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
  named_sync(kBarQ, kQThreads);
  for (int k = n - 2; k >= 0; --k) {
    const double2 tk = tau[k];
    if (tk.x == 0.0 && tk.y == 0.0) continue;
    const int m = n - k - 1;
    // s_j = tau v^H Q[k+1:, j]
    for (int j = t; j < m; j += kQThreads) {
      double2 s = make_double2(0.0, 0.0);
      for (int i = 0; i < m; ++i) {
        const double2 c = cmulc(A[(size_t)(k + 1 + i) * lda + k], Qm[(size_t)(k + 1 + i) * lda + k + 1 + j]);
        s.x += c.x; s.y += c.y;
      }
      sv[j] = cmul(tk, s);
    }
    named_sync(kBarQ, kQThreads);
    for (int idx = t; idx < m * m; idx += kQThreads) {
      const int i = idx / m, j = idx - i * m;
      const double2 c = cmul(A[(size_t)(k + 1 + i) * lda + k], sv[j]);
      double2& q = Qm[(size_t)(k + 1 + i) * lda + k + 1 + j];
      q.x -= c.x;
      q.y -= c.y;
    }
    named_sync(kBarQ, kQThreads);
  }
}

// ---- df64 complex numbers (re, im), stored as float4 (re.h, re.l, im.h, im.l):
// the same 16 bytes as an FP64 complex entry.
struct dc {
  dw re, im;
};
__device__ __forceinline__ dc dc_ld(const float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ float4 dc_st(dc a) { return make_float4(a.re.h, a.re.l, a.im.h, a.im.l); }
__device__ __forceinline__ dc dc_zero() { return {{0.0f, 0.0f}, {0.0f, 0.0f}}; }
__device__ __forceinline__ dc dc_add(dc a, dc b) { return {dw_add(a.re, b.re), dw_add(a.im, b.im)}; }
__device__ __forceinline__ dc dc_sub(dc a, dc b) { return {dw_sub(a.re, b.re), dw_sub(a.im, b.im)}; }
__device__ __forceinline__ dc dc_mul(dc a, dc b) {
  return {dw_sub(dw_mul(a.re, b.re), dw_mul(a.im, b.im)), dw_add(dw_mul(a.re, b.im), dw_mul(a.im, b.re))};
}
__device__ __forceinline__ dc dc_mulc(dc a, dc b) {   // conj(a) * b
  return {dw_add(dw_mul(a.re, b.re), dw_mul(a.im, b.im)), dw_sub(dw_mul(a.re, b.im), dw_mul(a.im, b.re))};
}

// Block sum of a df64 complex value; every thread gets the same sum (the
// warps' partials are added in warp order).
__device__ dc block_sum_dc(dc v, float4* red) {
  for (int o = 16; o > 0; o >>= 1) {
    dc u;
    u.re.h = __shfl_xor_sync(0xffffffffu, v.re.h, o);
    u.re.l = __shfl_xor_sync(0xffffffffu, v.re.l, o);
    u.im.h = __shfl_xor_sync(0xffffffffu, v.im.h, o);
    u.im.l = __shfl_xor_sync(0xffffffffu, v.im.l, o);
    v = dc_add(v, u);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = dc_st(v);
  __syncthreads();
  dc t = dc_ld(red[0]);
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i) t = dc_add(t, dc_ld(red[i]));
  return t;
}

// Step 1 in df64 for the non-FP64 plans: the same reflectors in the same
// order as the FP64 form, on A scaled by the power of two sc that brings
// max |A_ij| into [1, 2) (df64 has the exponent range of FP32).  FP64 is the
// scarce pipe on this part, and the reduction's products and its reductions'
// dependent adds were the longest phase of the solver in FP64.  On return d
// and e hold the tridiagonal (FP64, unscaled; e[n-1] is the caller's), and
// the reflectors below the subdiagonal of A and tau are FP64 complex, as the
// Q-forming warps read them.  A coefficient column whose |alpha|^2 + |x|^2 is
// below 2^-120 (entries below about 1e-18 of max |A_ij|) is left unreflected,
// a perturbation far below the arithmetic's 2^-47.
__device__ void householder_dw(const double2* __restrict__ G, double2* A, int lda, int n, double2* tau,
                               double2* pv, double2* vv, double2* part, double* d, double* e, double2* red) {
  const int tid = threadIdx.x, nth = blockDim.x;
  float4* A4 = reinterpret_cast<float4*>(A);
  float4* tau4 = reinterpret_cast<float4*>(tau);
  float4* pv4 = reinterpret_cast<float4*>(pv);
  float4* vv4 = reinterpret_cast<float4*>(vv);
  float4* part4 = reinterpret_cast<float4*>(part);
  float4* red4 = reinterpret_cast<float4*>(red);
  double amax = 0.0;
  for (int i = tid; i < n * n; i += nth) {
    const double2 g = G[i];
    amax = fmax(amax, fmax(fabs(g.x), fabs(g.y)));
  }
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((tid & 31) == 0) red[tid >> 5].x = amax;
  __syncthreads();
  amax = 0.0;
  for (int i = 0; i < (nth >> 5); ++i) amax = fmax(amax, red[i].x);
  const double sc = amax > 0.0 ? scalbn(1.0, -ilogb(amax)) : 1.0;
  for (int i = tid; i < n * n; i += nth) {
    const int r = i / n, c = i - r * n;
    const double2 g = G[i];
    const dw re = dw_from_double(g.x * sc), im = dw_from_double(g.y * sc);
    A4[(size_t)r * lda + c] = make_float4(re.h, re.l, im.h, im.l);
  }
  __syncthreads();
  for (int k = 0; k + 1 < n; ++k) {
    const int m = n - k - 1;
    // alpha and x are read before the barriers of the sum below, after
    // which the column is overwritten by v
    const dc alpha = dc_ld(A4[(size_t)(k + 1) * lda + k]);
    dc pt = dc_zero();
    for (int i = 1 + tid; i < m; i += nth) {
      const dc x = dc_ld(A4[(size_t)(k + 1 + i) * lda + k]);
      pt.re = dw_add(pt.re, dw_add(dw_mul(x.re, x.re), dw_mul(x.im, x.im)));
    }
    const dw xn2 = block_sum_dc(pt, red4).re;     // |x[1:]|^2, the same in every thread
    // the reflector, computed by every thread from the same operands (no broadcast)
    dc t = dc_zero(), scale = dc_zero();
    dw beta = alpha.re;                            // stays alpha when no reflection is needed
    {
      const dw a2 = dw_add(dw_add(dw_mul(alpha.re, alpha.re), dw_mul(alpha.im, alpha.im)), xn2);
      if ((xn2.h > 0.0f || alpha.im.h != 0.0f) && a2.h > 0x1p-120f) {
        const dw nrm = dw_mul(a2, dw_rsqrt(a2));
        beta = alpha.re.h >= 0.0f ? dw_neg(nrm) : nrm;
        t.re = dw_div(dw_sub(beta, alpha.re), beta);
        t.im = dw_div(dw_neg(alpha.im), beta);
        // scale = 1 / (alpha - beta)
        const dc den = {dw_sub(alpha.re, beta), alpha.im};
        const dw dd2 = dw_add(dw_mul(den.re, den.re), dw_mul(den.im, den.im));
        scale.re = dw_div(den.re, dd2);
        scale.im = dw_neg(dw_div(den.im, dd2));
      }
    }
    if (tid == 0) {
      tau4[k] = dc_st(t);
      e[k] = dw_to_double(beta) / sc;
    }
    if (t.re.h == 0.0f && t.im.h == 0.0f) continue;
    // v = (1, x[1:] * scale): in place below the subdiagonal and in vv
    for (int i = tid; i < m; i += nth) {
      float4* a = A4 + (size_t)(k + 1 + i) * lda + k;
      const dc v = i == 0 ? dc{{1.0f, 0.0f}, {0.0f, 0.0f}} : dc_mul(dc_ld(*a), scale);
      *a = dc_st(v);
      vv4[i] = dc_st(v);
    }
    __syncthreads();
    // p = tau * A22 v (A22 Hermitian: columns read), S partial sums per i in a fixed order
    const int S = max(1, min(8, nth / m));
    if (tid < S * m) {
      const int i = tid % m, sidx = tid / m;
      dc acc = dc_zero();
      for (int j = sidx; j < m; j += S)
        acc = dc_add(acc, dc_mulc(dc_ld(A4[(size_t)(k + 1 + j) * lda + (k + 1 + i)]), dc_ld(vv4[j])));
      part4[sidx * m + i] = dc_st(acc);
    }
    __syncthreads();
    // p_i and p^H v; then w = p - (tau/2) (p^H v) v, each thread on the i it formed
    dc dot = dc_zero();
    for (int i = tid; i < m; i += nth) {
      dc acc = dc_ld(part4[i]);
      for (int q = 1; q < S; ++q) acc = dc_add(acc, dc_ld(part4[q * m + i]));
      const dc pi = dc_mul(t, acc);
      pv4[i] = dc_st(pi);
      dot = dc_add(dot, dc_mulc(pi, dc_ld(vv4[i])));
    }
    dot = block_sum_dc(dot, red4);
    const dc half_t = {{-0.5f * t.re.h, -0.5f * t.re.l}, {-0.5f * t.im.h, -0.5f * t.im.l}};   // exact
    const dc al = dc_mul(half_t, dot);
    for (int i = tid; i < m; i += nth) pv4[i] = dc_st(dc_add(dc_ld(pv4[i]), dc_mul(al, dc_ld(vv4[i]))));
    __syncthreads();
    // A22 -= v w^H + w v^H
    for (int idx = tid; idx < m * m; idx += nth) {
      const int i = idx / m, j = idx - i * m;
      const dc vi = dc_ld(vv4[i]), vj = dc_ld(vv4[j]);
      const dc wi = dc_ld(pv4[i]), wj = dc_ld(pv4[j]);
      float4* a = A4 + (size_t)(k + 1 + i) * lda + (k + 1 + j);
      // v_i conj(w_j) + w_i conj(v_j)
      *a = dc_st(dc_sub(dc_ld(*a), dc_add(dc_mulc(wj, vi), dc_mulc(vj, wi))));
    }
    __syncthreads();
  }
  // the diagonal, then the reflectors (strictly below it) and tau to FP64 in place
  for (int i = tid; i < n; i += nth) {
    const float4 a = A4[(size_t)i * lda + i];
    d[i] = ((double)a.x + (double)a.y) / sc;
  }
  for (int idx = tid; idx < n * n; idx += nth) {
    const int r = idx / n, c = idx - r * n;
    if (r > c) {
      const float4 a = A4[(size_t)r * lda + c];
      A[(size_t)r * lda + c] = make_double2((double)a.x + (double)a.y, (double)a.z + (double)a.w);
    }
  }
  for (int k = tid; k + 1 < n; k += nth) {
    const float4 t4 = tau4[k];
    tau[k] = make_double2((double)t4.x + (double)t4.y, (double)t4.z + (double)t4.w);
  }
}

template <bool kDW>
__global__ void __launch_bounds__(kThreads, 2) k_eig_tridiag(const double* __restrict__ gram, int n,
                                                          double* __restrict__ lam, double* __restrict__ psi,
                                                          double* __restrict__ gws, unsigned* __restrict__ flags,
                                                          int max_iter) {
  const int f = blockIdx.x;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int warp = tid >> 5;
  const int lda = odd_stride(n);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* red = reinterpret_cast<double2*>(smem_raw);          // [32]
  double2* tau = red + 32;                                       // [n]
  double2* pv = tau + n;                                         // [n] p / w; later s of form_q
  double2* vv = pv + n;                                          // [n] reflector, contiguous
  double2* part = vv + n;                                        // [kThreads] matrix-vector partial sums
  double* d = reinterpret_cast<double*>(part + kThreads);        // [n]
  double* e = d + n;                                             // [n]
  double* rc = e + n;                                            // [2][n] rotation cosines
  double* rsn = rc + 2 * n;                                      // [2][n] rotation sines
  int* ctl = reinterpret_cast<int*>(rsn + 2 * n);                // [8] control words
  // per frequency: A [n][lda] complex (reflectors, then V), Q [n][lda] complex, Z [n][lda] real
  double2* A;
  {
    uint8_t* after = reinterpret_cast<uint8_t*>(ctl + 8);
    after = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(after) + 15) & ~uintptr_t(15));
    // per-frequency stride rounded up to an even number of doubles: double2 needs 16-byte alignment
    const size_t stride = ((size_t)5 * n * lda + 1) & ~(size_t)1;
    A = (n <= kEigSmemMaxNb) ? reinterpret_cast<double2*>(after) : reinterpret_cast<double2*>(gws + (size_t)f * stride);
  }
  double2* Qm = A + (size_t)n * lda;
  double* Z = reinterpret_cast<double*>(Qm + (size_t)n * lda);
  const double2* G = reinterpret_cast<const double2*>(gram) + (size_t)f * n * n;

  // ---------------- 1. Householder reduction to real tridiagonal form
  if constexpr (kDW) {
    householder_dw(G, A, lda, n, tau, pv, vv, part, d, e, red);
  } else {
    for (int i = tid; i < n * n; i += nth) {
      const int r = i / n, c = i - r * n;
      A[(size_t)r * lda + c] = G[i];
    }
    __syncthreads();
    for (int k = 0; k + 1 < n; ++k) {
      const int m = n - k - 1;                    // length of x = A[k+1:, k]
      double2 pt = make_double2(0.0, 0.0);
      for (int i = 1 + tid; i < m; i += nth) {
        const double2 x = A[(size_t)(k + 1 + i) * lda + k];
        pt.x += x.x * x.x + x.y * x.y;
      }
      const double xn2 = block_sum2(pt, red).x;   // |x[1:]|^2
      if (tid == 0) {
        const double2 alpha = A[(size_t)(k + 1) * lda + k];
        double2 t = make_double2(0.0, 0.0);
        double beta = alpha.x;                     // stays alpha when no reflection is needed
        double2 scale = make_double2(0.0, 0.0);
        if (xn2 > 0.0 || alpha.y != 0.0) {
          const double nrm = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2);
          beta = alpha.x >= 0.0 ? -nrm : nrm;
          t = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
          // scale = 1 / (alpha - beta)
          const double2 den = make_double2(alpha.x - beta, alpha.y);
          const double dd2 = den.x * den.x + den.y * den.y;
          scale = make_double2(den.x / dd2, -den.y / dd2);
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
      // v = (1, x[1:] * scale): stored in place below the subdiagonal and in vv
      for (int i = tid; i < m; i += nth) {
        double2* a = A + (size_t)(k + 1 + i) * lda + k;
        const double2 v = i == 0 ? make_double2(1.0, 0.0) : cmul(*a, scale);
        *a = v;
        vv[i] = v;
      }
      __syncthreads();
      // p = tau * A22 v with A22 Hermitian: p_i = tau sum_j conj(A22[j][i]) v_j,
      // S partial sums per i over j = s, s + S, ... (consecutive threads read
      // consecutive columns), added in a fixed order
      const int S = max(1, min(8, nth / m));
      if (tid < S * m) {
        const int i = tid % m, sidx = tid / m;
        double2 acc = make_double2(0.0, 0.0);
        for (int j = sidx; j < m; j += S) {
          const double2 c = cmulc(A[(size_t)(k + 1 + j) * lda + (k + 1 + i)], vv[j]);
          acc.x += c.x; acc.y += c.y;
        }
        part[sidx * m + i] = acc;
      }
      __syncthreads();
      for (int i = tid; i < m; i += nth) {
        double2 acc = part[i];
        for (int q = 1; q < S; ++q) { acc.x += part[q * m + i].x; acc.y += part[q * m + i].y; }
        pv[i] = cmul(t, acc);
      }
      __syncthreads();
      // w = p - (tau/2) (p^H v) v
      double2 dot = make_double2(0.0, 0.0);
      for (int i = tid; i < m; i += nth) {
        const double2 c = cmulc(pv[i], vv[i]);
        dot.x += c.x; dot.y += c.y;
      }
      dot = block_sum2(dot, red);
      const double2 al = cmul(make_double2(-0.5 * t.x, -0.5 * t.y), dot);
      __syncthreads();
      for (int i = tid; i < m; i += nth) {
        const double2 c = cmul(al, vv[i]);
        pv[i] = make_double2(pv[i].x + c.x, pv[i].y + c.y);
      }
      __syncthreads();
      // A22 -= v w^H + w v^H
      for (int idx = tid; idx < m * m; idx += nth) {
        const int i = idx / m, j = idx - i * m;
        const double2 vi = vv[i], vj = vv[j];
        const double2 wi = pv[i], wj = pv[j];
        double2& a = A[(size_t)(k + 1 + i) * lda + (k + 1 + j)];
        // v_i conj(w_j) + w_i conj(v_j)
        a.x -= (vi.x * wj.x + vi.y * wj.y) + (wi.x * vj.x + wi.y * vj.y);
        a.y -= (vi.y * wj.x - vi.x * wj.y) + (wi.y * vj.x - wi.x * vj.y);
      }
      __syncthreads();
    }
    for (int i = tid; i < n; i += nth) d[i] = A[(size_t)i * lda + i].x;
  }
  for (int idx = tid; idx < n * n; idx += nth) {
    const int r = idx / n, c = idx - r * n;
    Z[(size_t)r * lda + c] = r == c ? 1.0 : 0.0;
  }
  if (tid == 0) {
    e[n - 1] = 0.0;
    ctl[0] = 0;   // not-converged flag
  }
  __syncthreads();

  // ---------------- 2. QL (warp 0) | Z updates (warps 1-2) | Q (warps 3-7)
  if (warp == 0) ql_producer<kDW>(d, e, n, rc, rsn, ctl, max_iter);
  else if (warp < 3) ql_applier<kDW>(Z, lda, n, rc, rsn, ctl);
  else form_q(A, Qm, lda, n, tau, pv);
  __syncthreads();
  if (tid == 0 && ctl[0]) atomicOr(flags, FLAG_NOTCONV);

  // ---------------- 3. V = Q Z (into A's storage)
  double2* V = A;
  for (int idx = tid; idx < n * n; idx += nth) {
    const int i = idx / n, j = idx - i * n;
    const double2* qr = Qm + (size_t)i * lda;
    double sx = 0.0, sy = 0.0;
    for (int q = 0; q < n; ++q) {
      const double z = Z[(size_t)q * lda + j];
      sx = fma(qr[q].x, z, sx);
      sy = fma(qr[q].y, z, sy);
    }
    V[(size_t)i * lda + j] = make_double2(sx, sy);
  }
  __syncthreads();

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
      const double2 v = V[(size_t)j * lda + i];
      const double m2 = v.x * v.x + v.y * v.y;
      nrm += m2;
      if (m2 > best) { best = m2; piv = j; }
    }
    const double2 pvv = V[(size_t)piv * lda + i];
    const double pm = hypot(pvv.x, pvv.y);
    const double inv = 1.0 / sqrt(nrm);
    const double2 ph = make_double2(pvv.x / pm * inv, -pvv.y / pm * inv);
    lam[(size_t)f * n + rank] = li;
    double2* out = reinterpret_cast<double2*>(psi) + (size_t)f * n * n;
    for (int j = 0; j < n; ++j) {
      double2 v = cmul(V[(size_t)j * lda + i], ph);
      if (j == piv) v.y = 0.0;
      out[j * n + rank] = v;
    }
  }
}

}  // namespace

size_t eig_tridiag_smem_bytes(int nb) {
  const size_t lda = (size_t)odd_stride(nb);
  size_t b = sizeof(double2) * (32 + 3 * (size_t)nb + kThreads) + sizeof(double) * 6 * (size_t)nb +
             8 * sizeof(int) + 16;
  if (nb <= kEigSmemMaxNb) b += sizeof(double) * 5 * (size_t)nb * lda;
  return b;
}

size_t eig_tridiag_gws_doubles(int nb, int nf) {
  // per frequency: A and Q (n x lda complex) and Z (n x lda real)
  return (size_t)nf * (((size_t)5 * nb * odd_stride(nb) + 1) & ~(size_t)1);
}

cudaError_t launch_eig_tridiag(const spod_plan_s& p, cudaStream_t s) {
  const size_t smem = eig_tridiag_smem_bytes(p.nb);
  auto kern = p.f64 ? k_eig_tridiag<false> : k_eig_tridiag<true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<p.nf, kThreads, smem, s>>>(p.d_gram, p.nb, p.d_lam, p.d_psi, p.d_eigws, p.d_flags,
                                    p.eig_max_iter > 0 ? p.eig_max_iter : kMaxIter);
  return cudaGetLastError();
}

}  // namespace spod
