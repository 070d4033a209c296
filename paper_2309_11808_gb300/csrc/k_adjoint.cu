// Adjoint of the fit for losses on eigenvalues (spod_backward).
//
// For simple eigenvalues d lambda_k = psi_k^H dM_f psi_k.  With
// g_fk = dL/d lambda_fk:
//   G_f = 2 kappa sum_k g_fk psi_k psi_k^H                        (k_adj_gmat)
//   R_f = W Qhat_f G_f  (M x nb; computed by the mode kernels with the
//         coefficient matrix G_f and sqrt(W) as the output scale, because the
//         stored Qhat already carries sqrt(W))
//   dL/dxt[l step + n][m] += c w_n Re( sum_{f < nf} R_f[m][l] e^{+2 pi i f n / nfft} )
// summed over the blocks holding snapshot t (overlap-add), then the mean
// projection dL/dX[t][m] = dL/dxt[t][m] - (1/nt) sum_t' dL/dxt[t'][m].
//
// k_adjoint: one CTA per tile of TP points walks the blocks l = 0..nb-1 in
// order.  Per block it builds, for each point pair (a, b), the Hermitian
// extension H[f] = (Rt[f] + conj Rt[(N-f) mod N]) / 2 (Rt = R on the one-sided
// bins, 0 elsewhere) whose inverse DFT is the real series above, packs
// H_a + i H_b into one complex sequence, runs the forward Stockham FFT on its
// conjugate, and adds c w_n (Re, -Im) into a shared-memory ring of nfft output
// rows.  Rows [l step, (l+1) step) are final after block l and are written out
// with the mean already subtracted: the mean is computed first from the spectra,
// since sum_n c w_n Re(R_f e^{+2 pi i f n/N}) = Re(R_f * Wc_f) with
// Wc_f = c sum_n w_n e^{+2 pi i f n / N}.  No atomics: the result is
// bit-reproducible.
#include <algorithm>

#include "fft_common.cuh"

namespace spod {
namespace {

using namespace fft;

// G_f[l'][l] = 2 kappa sum_k g[f][k] psi[l'][k] conj(psi[l][k])  (compute type, interleaved complex),
// rows of ncol columns; with ncol = nb + 1 the last column is Wc_f sum_l G_f[l'][l], so
// that the mode kernel's extra output column is Wc_f sum_l R_f[m][l], the per-bin term of
// the mean of dL/dxt (sum over blocks and window samples of one column).
template <typename R>
__global__ void k_adj_gmat(const double* __restrict__ g, const double* __restrict__ psi, int nb, int ncol,
                           double two_kappa, const double* __restrict__ what, R* __restrict__ gmat) {
  const int f = blockIdx.x;
  const double2* P = reinterpret_cast<const double2*>(psi) + (size_t)f * nb * nb;
  // the extra column: sum_l G[l'][l] = 2 kappa sum_k g_k psi[l'][k] s_k, s_k = sum_l conj(psi[l][k])
  __shared__ double2 sk[256];
  if (ncol > nb) {
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
      double sr = 0.0, si = 0.0;
      for (int l = 0; l < nb; ++l) {
        sr += P[l * nb + k].x;
        si -= P[l * nb + k].y;
      }
      sk[k] = make_double2(sr, si);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * ncol; e += blockDim.x) {
    const int lp = e / ncol, l = e - lp * ncol;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < nb; ++k) {
      const double gk = g[(size_t)f * nb + k];
      const double2 a = P[lp * nb + k];
      // a * conj(psi[l][k]), or a * s_k for the extra column
      const double2 b = l < nb ? make_double2(P[l * nb + k].x, -P[l * nb + k].y) : sk[k];
      re += gk * (a.x * b.x - a.y * b.y);
      im += gk * (a.x * b.y + a.y * b.x);
    }
    re *= two_kappa;
    im *= two_kappa;
    if (l == nb) {
      const double wr = what[2 * f], wi = -what[2 * f + 1];   // Wc_f = conj(What_f)
      const double tr = re * wr - im * wi, ti = re * wi + im * wr;
      re = tr;
      im = ti;
    }
    R* o = gmat + ((size_t)f * nb * ncol + e) * 2;
    o[0] = (R)re;
    o[1] = (R)im;
  }
}

struct AdjArgs {
  int64_t M, m0, mcount, nt;
  int64_t roff;                      // point of R's first column
  int nfft, step, nb, nf;
  int ncol;                          // R columns per bin: nb, or nb + 1 (column nb: Wc_f sum_l R_f[.][l])
  int subtract_mean;
  double inv_nt;
  FftPlan fp;
};

template <typename R, int TP>
__global__ void __launch_bounds__(256) k_adjoint(const typename C2<R>::T* __restrict__ Rsp,  // [nf][nb][M]
                                                 int64_t rs, const R* __restrict__ win,
                                                 const typename C2<R>::T* __restrict__ tw_g,   // forward twiddles
                                                 const typename C2<R>::T* __restrict__ wc_g,   // Wc_f
                                                 R* __restrict__ dX, AdjArgs a) {
  using V = typename C2<R>::T;
  constexpr int C = TP / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.nfft, S = a.step;
  V* bufA = reinterpret_cast<V*>(smem_raw);                 // [N][C]
  V* bufB = bufA + (size_t)N * C;
  V* tw = bufB + (size_t)N * C;                             // [N] forward twiddles
  V* wc = tw + N;                                           // [nf]
  R* ring = reinterpret_cast<R*>(wc + a.nf);                // [N][TP] overlap-add accumulator
  R* mean = ring + (size_t)N * TP;                          // [TP]
  R* red = mean + TP;                                       // [256] reduction scratch

  const int64_t lm0 = (int64_t)blockIdx.x * TP;
  const int64_t gm0 = a.m0 + lm0;                           // global point (dX)
  const int64_t rm0 = gm0 - a.roff;                         // column in R
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += blockDim.x) tw[i] = tw_g[i];
  for (int i = tid; i < a.nf; i += blockDim.x) wc[i] = wc_g[i];
  for (int i = tid; i < N * TP; i += blockDim.x) ring[i] = (R)0;
  __syncthreads();

  // ---- mean of dL/dxt per point: (1/nt) sum_l Re(sum_f R[f][l][m] Wc_f), from
  // R's extra column when it has one
  {
    const int p = tid % TP;
    const int q = tid / TP;                 // 0 .. 256/TP - 1
    constexpr int Q = 256 / TP;
    R acc = 0;
    if (lm0 + p < a.mcount) {
      if (a.ncol > a.nb) {
        for (int f = q; f < a.nf; f += Q) acc += Rsp[((int64_t)f * a.ncol + a.nb) * rs + rm0 + p].x;
      } else {
        for (int e = q; e < a.nb * a.nf; e += Q) {
          const int l = e / a.nf, f = e - l * a.nf;
          const V r = Rsp[((int64_t)f * a.ncol + l) * rs + rm0 + p];
          const V w = wc[f];
          acc += r.x * w.x - r.y * w.y;
        }
      }
    }
    red[tid] = acc;
    __syncthreads();
    if (tid < TP) {
      R s = 0;
      for (int k = 0; k < Q; ++k) s += red[tid + k * TP];
      mean[tid] = a.subtract_mean ? (R)(s * (R)a.inv_nt) : (R)0;
    }
    __syncthreads();
  }

  auto write_rows = [&](int64_t t0, int64_t t1) {
    // rows [t0, t1) of this tile: ring value minus the mean; the ring rows are cleared
    for (int64_t idx = tid; idx < (t1 - t0) * TP; idx += blockDim.x) {
      const int64_t t = t0 + idx / TP;
      const int p = (int)(idx % TP);
      const int slot = (int)(t % N);
      R v = ring[slot * TP + p];
      ring[slot * TP + p] = (R)0;
      if (lm0 + p < a.mcount) dX[t * a.M + gm0 + p] = v - mean[p];
    }
  };

  for (int l = 0; l < a.nb; ++l) {
    // ---- conj of the packed Hermitian extension: conj(H_a + i H_b) for each column
    // pair, H[f] = Rt[f] + conj Rt[(N - f) mod N] with Rt = R on the one-sided bins
    // and 0 elsewhere.  Each R value is read once: a bin f of the one-sided range
    // gives entry f and, for 0 < f < N - f, the mirror entry N - f (whose H is
    // conj R[f]); the bins f with N - f < nf as well (f = 0, N/2) are their own
    // mirrors.
    for (int idx = tid; idx < a.nf * C; idx += blockDim.x) {
      const int f = idx / C, j = idx - f * C;
      const int fm = (f == 0) ? 0 : N - f;
      V ra = mk<R>(0, 0), rb = mk<R>(0, 0);
      const int64_t pa = lm0 + 2 * j;       // local index (bounds)
      const int64_t ga = rm0 + 2 * j;       // column in R
      if (pa < a.mcount) ra = Rsp[((int64_t)f * a.ncol + l) * rs + ga];
      if (pa + 1 < a.mcount) rb = Rsp[((int64_t)f * a.ncol + l) * rs + ga + 1];
      // Y = (ha + i hb) / 2 ; store conj(Y)
      auto put = [&](int e, V ha, V hb) {
        const R yr = (R)0.5 * (ha.x - hb.y), yi = (R)0.5 * (ha.y + hb.x);
        bufA[e * C + j] = mk<R>(yr, -yi);
      };
      if (fm < a.nf) {                       // f = 0 or f = N/2: H = R + conj R
        put(f, mk<R>(ra.x + ra.x, (R)0), mk<R>(rb.x + rb.x, (R)0));
      } else {
        put(f, ra, rb);                                      // H[f] = R[f]
        put(fm, mk<R>(ra.x, -ra.y), mk<R>(rb.x, -rb.y));     // H[N - f] = conj R[f]
      }
    }
    // (the entries written cover 0 .. N-1 once each, for even and odd N)
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
    // ---- y = conj(FFT(conj Y)): point a = Re, point b = -Im ; window, overlap-add
    const int64_t tb = (int64_t)l * S;
    for (int idx = tid; idx < N * C; idx += blockDim.x) {
      const int n = idx / C, j = idx - n * C;
      const V z = src[n * C + j];
      const R cw = win[n];
      const int slot = (int)((tb + n) % N);
      ring[slot * TP + 2 * j] += cw * z.x;
      ring[slot * TP + 2 * j + 1] += -cw * z.y;
    }
    __syncthreads();
    // rows finished by this block
    write_rows(tb, tb + S);
    __syncthreads();
  }
  // the last block's remaining rows, then the uncovered tail (gradient 0 before projection)
  const int64_t tdone = (int64_t)a.nb * S;
  const int64_t tcov = (int64_t)(a.nb - 1) * S + N;
  write_rows(tdone, tcov);
  __syncthreads();
  for (int64_t idx = tid; idx < (a.nt - tcov) * TP; idx += blockDim.x) {
    const int64_t t = tcov + idx / TP;
    const int p = (int)(idx % TP);
    if (lm0 + p < a.mcount) dX[t * a.M + gm0 + p] = -mean[p];
  }
}

// ---------------------------------------------------------------- nfft = 512, FP32
// The same adjoint with the transform in two register passes (n = k1 + 16 k2,
// 16-point DFTs in registers, the last radix-2 step exchanged between the two
// threads of a pair by shuffles) instead of the generic Stockham passes:
// thread (column, k1, h) ends with 16 time samples of its column, windows
// them and adds them into the overlap-add ring directly.  TP = 16 points
// (8 column pairs) per CTA, 256 threads.
constexpr int kAdjTP = 16;
constexpr int kAdjC = kAdjTP / 2;
constexpr int kAdjN = 512;

__device__ __forceinline__ float2 adj_cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// 16-point forward DFT in registers (radix 4 x 4).
__device__ __forceinline__ void adj_dft16(float2* v) {
  constexpr float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, r2 = 0.70710678118654752440f;
  float2 a[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float2 t[4] = {v[q], v[q + 4], v[q + 8], v[q + 12]};
    dft_small<4, float2, float>(t);
#pragma unroll
    for (int r = 0; r < 4; ++r) a[q][r] = t[r];
  }
  const float2 w1 = make_float2(c1, -s1), w3 = make_float2(s1, -c1), w9 = make_float2(-c1, s1);
  a[1][1] = adj_cmul(a[1][1], w1);
  a[1][2] = make_float2(r2 * (a[1][2].x + a[1][2].y), r2 * (a[1][2].y - a[1][2].x));
  a[1][3] = adj_cmul(a[1][3], w3);
  a[2][1] = make_float2(r2 * (a[2][1].x + a[2][1].y), r2 * (a[2][1].y - a[2][1].x));
  a[2][2] = mul_mi(a[2][2]);
  a[2][3] = make_float2(r2 * (a[2][3].y - a[2][3].x), -r2 * (a[2][3].x + a[2][3].y));
  a[3][1] = adj_cmul(a[3][1], w3);
  a[3][2] = make_float2(r2 * (a[3][2].y - a[3][2].x), -r2 * (a[3][2].x + a[3][2].y));
  a[3][3] = adj_cmul(a[3][3], w9);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    float2 t[4] = {a[0][r], a[1][r], a[2][r], a[3][r]};
    dft_small<4, float2, float>(t);
#pragma unroll
    for (int q = 0; q < 4; ++q) v[r + 4 * q] = t[q];
  }
}

__global__ void __launch_bounds__(256, 2) k_adjoint512(const float2* __restrict__ Rsp, int64_t rs,
                                                       const float* __restrict__ win,
                                                       const float2* __restrict__ tw_g,
                                                       const float2* __restrict__ wc_g, float* __restrict__ dX,
                                                       AdjArgs a) {
  constexpr int N = kAdjN, TP = kAdjTP, C = kAdjC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int S = a.step;
  float2* bufA = reinterpret_cast<float2*>(smem_raw);        // [N][C]  conj(Y)
  float2* bufB = bufA + (size_t)N * C;                       // [N][C]  pass A output
  float2* tw = bufB + (size_t)N * C;                         // [N]
  float2* wc = tw + N;                                       // [nf]
  float* ring = reinterpret_cast<float*>(wc + a.nf);         // [N][TP]
  float* mean = ring + (size_t)N * TP;                       // [TP]
  float* red = mean + TP;                                    // [256]

  const int64_t lm0 = (int64_t)blockIdx.x * TP;
  const int64_t gm0 = a.m0 + lm0;
  const int64_t rm0 = gm0 - a.roff;
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += blockDim.x) tw[i] = tw_g[i];
  for (int i = tid; i < a.nf; i += blockDim.x) wc[i] = wc_g[i];
  for (int i = tid; i < N * TP; i += blockDim.x) ring[i] = 0.f;
  __syncthreads();

  // ---- mean of dL/dxt per point: (1/nt) sum_l Re(sum_f R[f][l][m] Wc_f)
  {
    const int p = tid % TP;
    const int q = tid / TP;
    constexpr int Q = 256 / TP;
    float acc = 0.f;
    if (lm0 + p < a.mcount) {
      if (a.ncol > a.nb) {
        for (int f = q; f < a.nf; f += Q) acc += Rsp[((int64_t)f * a.ncol + a.nb) * rs + rm0 + p].x;
      } else {
        for (int e = q; e < a.nb * a.nf; e += Q) {
          const int l = e / a.nf, f = e - l * a.nf;
          const float2 r = Rsp[((int64_t)f * a.ncol + l) * rs + rm0 + p];
          const float2 w = wc[f];
          acc = fmaf(r.x, w.x, acc);
          acc = fmaf(-r.y, w.y, acc);
        }
      }
    }
    red[tid] = acc;
    __syncthreads();
    if (tid < TP) {
      float sm = 0.f;
      for (int k = 0; k < Q; ++k) sm += red[tid + k * TP];
      mean[tid] = a.subtract_mean ? (float)(sm * a.inv_nt) : 0.f;
    }
    __syncthreads();
  }

  auto write_rows = [&](int64_t t0, int64_t t1) {
    for (int64_t idx = tid; idx < (t1 - t0) * TP; idx += blockDim.x) {
      const int64_t t = t0 + idx / TP;
      const int p = (int)(idx % TP);
      const int slot = (int)(t % N);
      const float v = ring[slot * TP + p];
      ring[slot * TP + p] = 0.f;
      if (lm0 + p < a.mcount) dX[t * a.M + gm0 + p] = v - mean[p];
    }
  };

  const int col = tid % C;
  const int jj = tid / C;                 // pass A: n2; pass B: 2 k1 + h
  // R of the next block is loaded into registers while the current block is
  // transformed (element it of thread tid: bin f, column pair j of idx = tid + 256 it)
  constexpr int kIt = ((kAdjN / 2 + 1) * C + 255) / 256;
  float2 pra[kIt], prb[kIt];
  auto load_block = [&](int l) {
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int idx = tid + 256 * it;
      const int f = idx / C, j = idx - f * C;
      float2 ra = make_float2(0.f, 0.f), rb = make_float2(0.f, 0.f);
      const int64_t pa = lm0 + 2 * j;
      const int64_t ga = rm0 + 2 * j;
      if (f < a.nf) {
        if (pa < a.mcount) ra = Rsp[((int64_t)f * a.ncol + l) * rs + ga];
        if (pa + 1 < a.mcount) rb = Rsp[((int64_t)f * a.ncol + l) * rs + ga + 1];
      }
      pra[it] = ra;
      prb[it] = rb;
    }
  };
  load_block(0);
  for (int l = 0; l < a.nb; ++l) {
    // ---- conj of the packed Hermitian extension (as in k_adjoint), from the
    // registers; then the next block's loads are issued
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int idx = tid + 256 * it;
      const int f = idx / C, j = idx - f * C;
      if (f >= a.nf) continue;
      const int fm = (f == 0) ? 0 : N - f;
      const float2 ra = pra[it], rb = prb[it];
      auto put = [&](int e, float2 ha, float2 hb) {
        const float yr = 0.5f * (ha.x - hb.y), yi = 0.5f * (ha.y + hb.x);
        bufA[e * C + j] = make_float2(yr, -yi);
      };
      if (fm < a.nf) {
        put(f, make_float2(ra.x + ra.x, 0.f), make_float2(rb.x + rb.x, 0.f));
      } else {
        put(f, ra, rb);
        put(fm, make_float2(ra.x, -ra.y), make_float2(rb.x, -rb.y));
      }
    }
    if (l + 1 < a.nb) load_block(l + 1);
    __syncthreads();
    // ---- pass A: n = 32 n1 + n2, thread (col, n2)
    {
      const int n2 = jj;
      float2 v[16];
#pragma unroll
      for (int n1 = 0; n1 < 16; ++n1) v[n1] = bufA[(32 * n1 + n2) * C + col];
      adj_dft16(v);
#pragma unroll
      for (int k1 = 1; k1 < 16; ++k1) v[k1] = adj_cmul(v[k1], tw[n2 * k1]);
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) bufB[(k1 * 32 + n2) * C + col] = v[k1];
    }
    __syncthreads();
    // ---- pass B: thread (col, k1, h) with the values n2 = 2 m + h; then the
    // radix-2 step with the partner thread (h ^ 1, lane tid ^ C), window and
    // overlap-add of its 16 samples n = k1 + 16 (k2 + 16 h)
    {
      const int k1 = jj >> 1, h = jj & 1;
      float2 v[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) v[m] = bufB[(k1 * 32 + 2 * m + h) * C + col];
      adj_dft16(v);
      const int64_t tb = (int64_t)l * S;
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        // h = 1 sends W32^k2 U_1, h = 0 sends U_0; each receives the other
        const float2 mine = h ? adj_cmul(v[k2], tw[16 * k2]) : v[k2];
        float2 other;
        other.x = __shfl_xor_sync(0xffffffffu, mine.x, C);
        other.y = __shfl_xor_sync(0xffffffffu, mine.y, C);
        const float2 z = h ? make_float2(other.x - mine.x, other.y - mine.y)
                           : make_float2(mine.x + other.x, mine.y + other.y);
        const int n = k1 + 16 * (k2 + 16 * h);
        const float cw = win[n];
        const int slot = (int)((tb + n) % N);
        float2* rp = reinterpret_cast<float2*>(ring + slot * TP + 2 * col);
        float2 acc = *rp;
        acc.x = fmaf(cw, z.x, acc.x);
        acc.y = fmaf(-cw, z.y, acc.y);
        *rp = acc;
      }
    }
    __syncthreads();
    write_rows((int64_t)l * S, (int64_t)(l + 1) * S);
    __syncthreads();
  }
  const int64_t tdone = (int64_t)a.nb * S;
  const int64_t tcov = (int64_t)(a.nb - 1) * S + N;
  write_rows(tdone, tcov);
  __syncthreads();
  for (int64_t idx = tid; idx < (a.nt - tcov) * TP; idx += blockDim.x) {
    const int64_t t = tcov + idx / TP;
    const int p = (int)(idx % TP);
    if (lm0 + p < a.mcount) dX[t * a.M + gm0 + p] = -mean[p];
  }
}

size_t adjoint512_smem_bytes(int nf) {
  return sizeof(float2) * ((size_t)2 * kAdjN * kAdjC + kAdjN + nf) +
         sizeof(float) * ((size_t)kAdjN * kAdjTP + kAdjTP + 256);
}

template <typename R>
cudaError_t launch_adjoint_t(const spod_plan_s& p, const void* d_R, int64_t rs, int64_t roff, int64_t m0,
                             int64_t mcount, void* d_dX, cudaStream_t s) {
  constexpr int TP = sizeof(R) == 8 ? 8 : 16;
  AdjArgs a;
  a.M = p.M; a.m0 = m0; a.mcount = mcount; a.nt = p.nt; a.roff = roff;
  a.nfft = p.nfft; a.step = p.step; a.nb = p.nb; a.nf = p.nf; a.ncol = p.adj_cols;
  a.subtract_mean = p.desc.subtract_mean;
  a.inv_nt = 1.0 / (double)p.nt;
  a.fp = p.fft;
  const size_t smem = adjoint_smem_bytes(p);
  auto kern = k_adjoint<R, TP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = (mcount + TP - 1) / TP;
  kern<<<(unsigned)grid, 256, smem, s>>>(static_cast<const typename C2<R>::T*>(d_R), rs,
                                         static_cast<const R*>(p.d_win), static_cast<const typename C2<R>::T*>(p.d_tw),
                                         static_cast<const typename C2<R>::T*>(p.d_wc), static_cast<R*>(d_dX), a);
  return cudaGetLastError();
}

}  // namespace

size_t adjoint_smem_bytes(const spod_plan_s& p) {
  const size_t R = p.f64 ? 8 : 4;
  const size_t TP = p.f64 ? 8 : 16;
  const size_t C = TP / 2;
  return 2 * R * ((size_t)p.nfft * C * 2 + p.nfft + p.nf) + R * ((size_t)p.nfft * TP + TP + 256);
}

cudaError_t launch_adj_gmat(const spod_plan_s& p, const double* d_g, cudaStream_t s) {
  // the extra column's Wc_f = conj(What_f), from the plan's FP64 What_f
  if (p.f64)
    k_adj_gmat<double><<<p.nf, 256, 0, s>>>(d_g, p.d_psi, p.nb, p.adj_cols, 2.0 * p.kappa, p.d_what,
                                             static_cast<double*>(p.d_bmat));
  else
    k_adj_gmat<float><<<p.nf, 256, 0, s>>>(d_g, p.d_psi, p.nb, p.adj_cols, 2.0 * p.kappa, p.d_what,
                                            static_cast<float*>(p.d_bmat));
  return cudaGetLastError();
}

cudaError_t launch_adjoint_chunk(const spod_plan_s& p, const void* d_R, int64_t rs, int64_t roff, int64_t m0,
                                 int64_t mcount, void* d_dX, cudaStream_t s) {
  if (!p.f64 && p.nfft == kAdjN) {
    AdjArgs a;
    a.M = p.M; a.m0 = m0; a.mcount = mcount; a.nt = p.nt; a.roff = roff;
    a.nfft = p.nfft; a.step = p.step; a.nb = p.nb; a.nf = p.nf; a.ncol = p.adj_cols;
    a.subtract_mean = p.desc.subtract_mean;
    a.inv_nt = 1.0 / (double)p.nt;
    a.fp = p.fft;
    const size_t smem = adjoint512_smem_bytes(p.nf);
    cudaError_t e = cudaFuncSetAttribute(k_adjoint512, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (mcount + kAdjTP - 1) / kAdjTP;
    k_adjoint512<<<(unsigned)grid, 256, smem, s>>>(static_cast<const float2*>(d_R), rs,
                                                   static_cast<const float*>(p.d_win),
                                                   static_cast<const float2*>(p.d_tw),
                                                   static_cast<const float2*>(p.d_wc), static_cast<float*>(d_dX), a);
    return cudaGetLastError();
  }
  return p.f64 ? launch_adjoint_t<double>(p, d_R, rs, roff, m0, mcount, d_dX, s)
               : launch_adjoint_t<float>(p, d_R, rs, roff, m0, mcount, d_dX, s);
}

}  // namespace spod
