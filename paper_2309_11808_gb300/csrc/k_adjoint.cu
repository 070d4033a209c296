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

// G_f[l'][l] = 2 kappa sum_k g[f][k] psi[l'][k] conj(psi[l][k])  (compute type, interleaved complex)
template <typename R>
__global__ void k_adj_gmat(const double* __restrict__ g, const double* __restrict__ psi, int nb, double two_kappa,
                           R* __restrict__ gmat) {
  const int f = blockIdx.x;
  const double2* P = reinterpret_cast<const double2*>(psi) + (size_t)f * nb * nb;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int lp = e / nb, l = e - lp * nb;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < nb; ++k) {
      const double gk = g[(size_t)f * nb + k];
      const double2 a = P[lp * nb + k], b = P[l * nb + k];
      // a * conj(b)
      re += gk * (a.x * b.x + a.y * b.y);
      im += gk * (a.y * b.x - a.x * b.y);
    }
    R* o = gmat + ((size_t)f * nb * nb + e) * 2;
    o[0] = (R)(two_kappa * re);
    o[1] = (R)(two_kappa * im);
  }
}

struct AdjArgs {
  int64_t M, m0, mcount, nt;
  int64_t roff;                      // point of R's first column
  int nfft, step, nb, nf;
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

  // ---- mean of dL/dxt per point: (1/nt) sum_l Re(sum_f R[f][l][m] Wc_f)
  {
    const int p = tid % TP;
    const int q = tid / TP;                 // 0 .. 256/TP - 1
    constexpr int Q = 256 / TP;
    R acc = 0;
    if (lm0 + p < a.mcount) {
      for (int e = q; e < a.nb * a.nf; e += Q) {
        const int l = e / a.nf, f = e - l * a.nf;
        const V r = Rsp[((int64_t)f * a.nb + l) * rs + rm0 + p];
        const V w = wc[f];
        acc += r.x * w.x - r.y * w.y;
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
      if (pa < a.mcount) ra = Rsp[((int64_t)f * a.nb + l) * rs + ga];
      if (pa + 1 < a.mcount) rb = Rsp[((int64_t)f * a.nb + l) * rs + ga + 1];
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

template <typename R>
cudaError_t launch_adjoint_t(const spod_plan_s& p, const void* d_R, int64_t rs, int64_t roff, int64_t m0,
                             int64_t mcount, void* d_dX, cudaStream_t s) {
  constexpr int TP = sizeof(R) == 8 ? 8 : 16;
  AdjArgs a;
  a.M = p.M; a.m0 = m0; a.mcount = mcount; a.nt = p.nt; a.roff = roff;
  a.nfft = p.nfft; a.step = p.step; a.nb = p.nb; a.nf = p.nf;
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
  if (p.f64)
    k_adj_gmat<double><<<p.nf, 256, 0, s>>>(d_g, p.d_psi, p.nb, 2.0 * p.kappa, static_cast<double*>(p.d_bmat));
  else
    k_adj_gmat<float><<<p.nf, 256, 0, s>>>(d_g, p.d_psi, p.nb, 2.0 * p.kappa, static_cast<float*>(p.d_bmat));
  return cudaGetLastError();
}

cudaError_t launch_adjoint_chunk(const spod_plan_s& p, const void* d_R, int64_t rs, int64_t roff, int64_t m0,
                                 int64_t mcount, void* d_dX, cudaStream_t s) {
  return p.f64 ? launch_adjoint_t<double>(p, d_R, rs, roff, m0, mcount, d_dX, s)
               : launch_adjoint_t<float>(p, d_R, rs, roff, m0, mcount, d_dX, s);
}

}  // namespace spod
