// Expansion coefficients and reconstruction ("SPOD for data compression",
// Eqs. coeffs and SPODrec):
//   A = (Phi_r^* W Phi_r)^{-1} Phi_r^* W Q,   Q~ = Phi_r A_r,
// Q = X^T - mu, over the leading nmodes_r modes of the selected one-sided bins
// and, for the bins other than DC and Nyquist, their complex conjugates (the
// modes of the negative frequencies, so that the set is closed under
// conjugation and the reconstruction of real data is real).
//
// The computation runs in the equivalent real basis: the complex span of
// {phi, conj phi} meets the real vectors in the real span of {Re phi, Im phi}
// (DC and Nyquist modes are real), so with the K real basis rows b_r
//   B = P_w X^T - P_w mu 1^T   (P_w rows W b_r; a plain GEMM over the M points),
//   G = P_w P_b^T               (P_b rows b_r; FP64 sums),
//   C = G^{-1} B,
// and a = c_re / 2 - i c_im / 2 for a conjugate pair (a = c_re at DC and
// Nyquist) recovers the complex coefficient of the mode at the positive bin
// (its conjugate bin carries conj(a)).  The reconstruction is
//   X~ = mu + P_b^T C  (real rows [nt][M]).
// The two large products run on k_gemm_simt, this file's SIMT GEMM (FP32 or
// FP64 as the plan; the product over the M points is split over CTAs and the
// parts summed in FP64 in a fixed order), as do C = G^{-1} B and the K x K
// Gram of the basis, its inverse and the packing.
#include <algorithm>
#include <vector>

#include "spod_internal.cuh"

namespace spod {
namespace {

struct BasisRow {
  int f, k, part;   // bin, mode, 0: Re phi, 1: Im phi
};

// P_w[r][m] = W_m b_r[m], P_b[r][m] = b_r[m]; phi is the interleaved complex
// mode array [nf][nmodes][M].
template <typename R>
__global__ void k_coeff_basis(const R* __restrict__ phi, int nmodes, int64_t M, const BasisRow* __restrict__ rows,
                              const R* __restrict__ sqrtW, R* __restrict__ Pw, R* __restrict__ Pb) {
  const int r = blockIdx.y;
  const BasisRow br = rows[r];
  const R* src = phi + ((int64_t)br.f * nmodes + br.k) * M * 2 + br.part;
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
    const R b = src[2 * m];
    const R sw = sqrtW[m];
    Pb[(int64_t)r * M + m] = b;
    Pw[(int64_t)r * M + m] = b * sw * sw;
  }
}

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

// G[i][j] = G[j][i] = sum_m P_w[i][m] P_b[j][m] (j >= i), and, for j == K,
// v[i] = sum_m P_w[i][m] mu[m]; FP64 sums in a fixed order.
template <typename R>
__global__ void k_coeff_gram(const R* __restrict__ Pw, const R* __restrict__ Pb, const double* __restrict__ mu,
                             int64_t M, int K, double* __restrict__ G, double* __restrict__ v) {
  __shared__ double red[32];
  const int i = blockIdx.x, j = blockIdx.y;
  if (j < K && j < i) return;
  const R* a = Pw + (int64_t)i * M;
  double acc = 0.0;
  if (j < K) {
    const R* b = Pb + (int64_t)j * M;
    for (int64_t m = threadIdx.x; m < M; m += blockDim.x) acc += (double)a[m] * (double)b[m];
  } else {
    for (int64_t m = threadIdx.x; m < M; m += blockDim.x) acc += (double)a[m] * mu[m];
  }
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) {
    if (j < K) {
      G[(int64_t)i * K + j] = t;
      G[(int64_t)j * K + i] = t;
    } else {
      v[i] = t;
    }
  }
}

// Ginv = G^{-1} for the symmetric positive definite G (K x K, FP64) by
// Gauss-Jordan elimination without pivoting (one CTA; G is overwritten).  A
// pivot that is not positive (a basis that is not linearly independent)
// raises FLAG_NOTCONV and leaves Ginv unusable.
__global__ void k_spd_inverse(double* __restrict__ G, double* __restrict__ Ginv, int K, unsigned* __restrict__ flags) {
  extern __shared__ double fac[];   // [K]
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int idx = tid; idx < K * K; idx += nth) Ginv[idx] = (idx / K == idx % K) ? 1.0 : 0.0;
  __syncthreads();
  for (int c = 0; c < K; ++c) {
    const double piv = G[(int64_t)c * K + c];
    if (!(piv > 0.0)) {
      if (tid == 0) atomicOr(flags, FLAG_NOTCONV);
      return;
    }
    __syncthreads();
    for (int j = tid; j < K; j += nth) {
      G[(int64_t)c * K + j] /= piv;
      Ginv[(int64_t)c * K + j] /= piv;
    }
    for (int i = tid; i < K; i += nth) fac[i] = G[(int64_t)i * K + c];
    __syncthreads();
    for (int idx = tid; idx < K * K; idx += nth) {
      const int i = idx / K, j = idx - i * K;
      if (i == c) continue;
      const double fi = fac[i];
      G[idx] -= fi * G[(int64_t)c * K + j];
      Ginv[idx] -= fi * Ginv[(int64_t)c * K + j];
    }
    __syncthreads();
  }
}

// d_A[q][t] (q = j * nmodes_r + k) from the real coefficients C (column-major
// K x nt): a = c[re] (DC, Nyquist) or c[re] / 2 - i c[im] / 2.
__global__ void k_coeff_pack(const double* __restrict__ C, const int2* __restrict__ qrows, int nq, int K,
                             int64_t nt, double2* __restrict__ A) {
  const int q = blockIdx.y;
  const int2 rr = qrows[q];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
    const double cre = C[t * K + rr.x];
    A[(int64_t)q * nt + t] = rr.y < 0 ? make_double2(cre, 0.0) : make_double2(0.5 * cre, -0.5 * C[t * K + rr.y]);
  }
}

// The real coefficients C (column-major K x nt, type R) from d_A.
template <typename R>
__global__ void k_coeff_unpack(const double2* __restrict__ A, const int2* __restrict__ qrows, int K, int64_t nt,
                               R* __restrict__ C) {
  const int q = blockIdx.y;
  const int2 rr = qrows[q];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = A[(int64_t)q * nt + t];
    if (rr.y < 0) {
      C[t * K + rr.x] = (R)a.x;
    } else {
      C[t * K + rr.x] = (R)(2.0 * a.x);
      C[t * K + rr.y] = (R)(-2.0 * a.y);
    }
  }
}

// Xrec[t][m] = mu[m].
template <typename R>
__global__ void k_fill_mean(const double* __restrict__ mu, int64_t M, int64_t n, R* __restrict__ X) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    X[e] = (R)mu[e % M];
}

// D(i, j) = beta D(i, j) + sum_k A(i, k) B(k, j) over the split's range of k,
// every operand given by element strides: A(i, k) = A[i sai + k sak],
// B(k, j) = B[k sbk + j sbj], D(i, j) = D[i sdi + j sdj].  64 x 64 tiles of D,
// 256 threads with 4 x 4 results each, k in steps of 16 staged in shared
// memory (loads along whichever index is contiguous).  Split z covers
// k in [z kper, (z + 1) kper) and writes D + z dsplit.
template <typename R>
__global__ void __launch_bounds__(256) k_gemm_simt(int ni, int nj, int64_t nk, const R* __restrict__ A, int64_t sai,
                                                   int64_t sak, const R* __restrict__ B, int64_t sbk, int64_t sbj,
                                                   R* __restrict__ D, int64_t sdi, int64_t sdj, int64_t dsplit,
                                                   R beta, int64_t kper) {
  constexpr int TI = 64, TJ = 64, TK = 16;
  __shared__ R As[TK][TI + 4];
  __shared__ R Bs[TK][TJ + 4];
  const int i0 = blockIdx.x * TI, j0 = blockIdx.y * TJ;
  const int64_t k0 = (int64_t)blockIdx.z * kper;
  const int64_t k1 = k0 + kper < nk ? k0 + kper : nk;
  R* Dz = D + (int64_t)blockIdx.z * dsplit;
  const int tid = threadIdx.x;
  // the output index that is contiguous in D varies fastest across threads
  const bool jfast = sdj == 1;
  const int ti = (jfast ? tid / 16 : tid % 16) * 4, tj = (jfast ? tid % 16 : tid / 16) * 4;
  R acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = (R)0;
  for (int64_t kb = k0; kb < k1; kb += TK) {
    for (int e = tid; e < TI * TK; e += 256) {
      const int kk = sak == 1 ? e % TK : e / TI, ii = sak == 1 ? e / TK : e % TI;
      const int gi = i0 + ii;
      const int64_t gk = kb + kk;
      As[kk][ii] = (gi < ni && gk < k1) ? A[(int64_t)gi * sai + gk * sak] : (R)0;
    }
    for (int e = tid; e < TK * TJ; e += 256) {
      const int kk = sbk == 1 ? e % TK : e / TJ, jj = sbk == 1 ? e / TK : e % TJ;
      const int gj = j0 + jj;
      const int64_t gk = kb + kk;
      Bs[kk][jj] = (gj < nj && gk < k1) ? B[gk * sbk + (int64_t)gj * sbj] : (R)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      R a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = As[kk][ti + q]; b[q] = Bs[kk][tj + q]; }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int gi = i0 + ti + x, gj = j0 + tj + y;
      if (gi < ni && gj < nj) {
        R* d = Dz + (int64_t)gi * sdi + (int64_t)gj * sdj;
        *d = beta == (R)0 ? acc[x][y] : beta * *d + acc[x][y];
      }
    }
}

// out[e] = sum_z parts[z][e] (FP64, z in order) - v[e % K]  (B - v 1^T, column-major K x nt)
template <typename R>
__global__ void k_coeff_center_parts(const R* __restrict__ parts, int nsplit, const double* __restrict__ v, int K,
                                     int64_t n, double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int z = 0; z < nsplit; ++z) acc += (double)parts[(int64_t)z * n + e];
    out[e] = acc - v[e % K];
  }
}

template <typename R>
cudaError_t gemm(int ni, int nj, int64_t nk, const R* A, int64_t sai, int64_t sak, const R* B, int64_t sbk,
                 int64_t sbj, R* D, int64_t sdi, int64_t sdj, R beta, int nsplit, int64_t dsplit, cudaStream_t s) {
  const int64_t kper = ((nk + nsplit - 1) / nsplit + 15) / 16 * 16;
  dim3 grid((unsigned)((ni + 63) / 64), (unsigned)((nj + 63) / 64), (unsigned)nsplit);
  k_gemm_simt<R><<<grid, 256, 0, s>>>(ni, nj, nk, A, sai, sak, B, sbk, sbj, D, sdi, sdj, dsplit, beta, kper);
  return cudaGetLastError();
}

bool self_conjugate(int f, int nfft) { return f == 0 || (nfft % 2 == 0 && f == nfft / 2); }

// Basis rows and, per (selected bin, mode), the rows of its real and
// imaginary parts (-1: none).
void basis_rows(const spod_plan_s& p, int nmodes_r, int nsel, const int* h_freqs, std::vector<BasisRow>* rows,
                std::vector<int2>* qrows) {
  for (int j = 0; j < nsel; ++j) {
    for (int k = 0; k < nmodes_r; ++k) {
      const int f = h_freqs[j];
      int2 q;
      q.x = (int)rows->size();
      rows->push_back({f, k, 0});
      q.y = -1;
      if (!self_conjugate(f, p.nfft)) {
        q.y = (int)rows->size();
        rows->push_back({f, k, 1});
      }
      qrows->push_back(q);
    }
  }
}

struct Scratch {
  std::vector<void*> ptrs;
  cudaStream_t s;
  cudaError_t err = cudaSuccess;
  void* get(size_t bytes) {
    void* q = nullptr;
    if (err == cudaSuccess) err = cudaMallocAsync(&q, bytes, s);
    if (err == cudaSuccess) ptrs.push_back(q);
    return q;
  }
  ~Scratch() {
    for (void* q : ptrs) cudaFreeAsync(q, s);
  }
};

// P_w, P_b (K x M, type R) of the selected modes.
template <typename R>
cudaError_t build_basis(const spod_plan_s& p, const void* d_Phi, int nmodes, const std::vector<BasisRow>& rows,
                        Scratch& sc, R** Pw, R** Pb, cudaStream_t s) {
  const int K = (int)rows.size();
  const int64_t M = p.M;
  BasisRow* d_rows = static_cast<BasisRow*>(sc.get(sizeof(BasisRow) * K));
  *Pw = static_cast<R*>(sc.get(sizeof(R) * (size_t)K * M));
  *Pb = static_cast<R*>(sc.get(sizeof(R) * (size_t)K * M));
  if (sc.err != cudaSuccess) return sc.err;
  cudaError_t e = cudaMemcpyAsync(d_rows, rows.data(), sizeof(BasisRow) * K, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)std::min<int64_t>((M + 255) / 256, 1024), (unsigned)K);
  k_coeff_basis<R><<<grid, 256, 0, s>>>(static_cast<const R*>(d_Phi), nmodes, M, d_rows,
                                        static_cast<const R*>(p.d_sqrtW), *Pw, *Pb);
  return cudaGetLastError();
}

template <typename R>
cudaError_t coeffs_t(spod_plan_s& p, const void* d_X, const void* d_Phi, int nmodes, int nmodes_r, int nsel,
                     const int* h_freqs, double* d_A, cudaStream_t s) {
  std::vector<BasisRow> rows;
  std::vector<int2> qrows;
  basis_rows(p, nmodes_r, nsel, h_freqs, &rows, &qrows);
  const int K = (int)rows.size();
  const int64_t M = p.M, nt = p.nt;
  Scratch sc;
  sc.s = s;
  R *Pw = nullptr, *Pb = nullptr;
  cudaError_t e = build_basis<R>(p, d_Phi, nmodes, rows, sc, &Pw, &Pb, s);
  if (e != cudaSuccess) return e;
  // the product over the M points, split so that the grid covers the GPU
  const int tiles = ((K + 63) / 64) * (int)((nt + 63) / 64);
  const int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>({64, (4 * p.num_sms + tiles - 1) / tiles, M / 1024}));
  R* B = static_cast<R*>(sc.get(sizeof(R) * (size_t)K * nt * nsplit));
  double* B64 = static_cast<double*>(sc.get(sizeof(double) * (size_t)K * nt));
  double* C = static_cast<double*>(sc.get(sizeof(double) * (size_t)K * nt));
  double* G = static_cast<double*>(sc.get(sizeof(double) * (size_t)K * K));
  double* Ginv = static_cast<double*>(sc.get(sizeof(double) * (size_t)K * K));
  double* v = static_cast<double*>(sc.get(sizeof(double) * K));
  int2* d_q = static_cast<int2*>(sc.get(sizeof(int2) * qrows.size()));
  if (sc.err != cudaSuccess) return sc.err;
  e = cudaMemcpyAsync(d_q, qrows.data(), sizeof(int2) * qrows.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  // G and v
  k_coeff_gram<R><<<dim3((unsigned)K, (unsigned)(K + 1)), 256, 0, s>>>(Pw, Pb, p.d_mu, M, K, G, v);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_spd_inverse<<<1, 1024, sizeof(double) * K, s>>>(G, Ginv, K, p.d_flags);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // B = P_w X^T (column-major K x nt; X[t][m]), per split of the points, then B - v 1^T in FP64
  e = gemm<R>(K, (int)nt, M, Pw, M, 1, static_cast<const R*>(d_X), 1, M, B, 1, K, (R)0, nsplit, (int64_t)K * nt, s);
  if (e != cudaSuccess) return e;
  k_coeff_center_parts<R><<<1024, 256, 0, s>>>(B, nsplit, v, K, (int64_t)K * nt, B64);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // C = G^{-1} (B - v 1^T)  (FP64, column-major K x nt)
  e = gemm<double>(K, (int)nt, K, Ginv, K, 1, B64, 1, K, C, 1, K, 0.0, 1, 0, s);
  if (e != cudaSuccess) return e;
  dim3 pg((unsigned)std::min<int64_t>((nt + 255) / 256, 1024), (unsigned)qrows.size());
  k_coeff_pack<<<pg, 256, 0, s>>>(C, d_q, (int)qrows.size(), K, nt, reinterpret_cast<double2*>(d_A));
  return cudaGetLastError();
}

template <typename R>
cudaError_t reconstruct_t(spod_plan_s& p, const void* d_Phi, int nmodes, int nmodes_r, int nsel, const int* h_freqs,
                          const double* d_A, void* d_Xrec, cudaStream_t s) {
  std::vector<BasisRow> rows;
  std::vector<int2> qrows;
  basis_rows(p, nmodes_r, nsel, h_freqs, &rows, &qrows);
  const int K = (int)rows.size();
  const int64_t M = p.M, nt = p.nt;
  Scratch sc;
  sc.s = s;
  R *Pw = nullptr, *Pb = nullptr;
  cudaError_t e = build_basis<R>(p, d_Phi, nmodes, rows, sc, &Pw, &Pb, s);
  if (e != cudaSuccess) return e;
  R* C = static_cast<R*>(sc.get(sizeof(R) * (size_t)K * nt));
  int2* d_q = static_cast<int2*>(sc.get(sizeof(int2) * qrows.size()));
  if (sc.err != cudaSuccess) return sc.err;
  e = cudaMemcpyAsync(d_q, qrows.data(), sizeof(int2) * qrows.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  dim3 pg((unsigned)std::min<int64_t>((nt + 255) / 256, 1024), (unsigned)qrows.size());
  k_coeff_unpack<R><<<pg, 256, 0, s>>>(reinterpret_cast<const double2*>(d_A), d_q, K, nt, C);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  R* X = static_cast<R*>(d_Xrec);
  k_fill_mean<R><<<2048, 256, 0, s>>>(p.d_mu, M, M * nt, X);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // X[t][m] += sum_r C[t][r] P_b[r][m]  (C column-major K x nt, P_b rows of M)
  return gemm<R>((int)nt, (int)M, K, C, K, 1, Pb, M, 1, X, M, 1, (R)1, 1, 0, s);
}

}  // namespace

int coeff_basis_size(const spod_plan_s& p, int nmodes_r, int nsel, const int* h_freqs) {
  int K = 0;
  for (int j = 0; j < nsel; ++j) K += nmodes_r * (self_conjugate(h_freqs[j], p.nfft) ? 1 : 2);
  return K;
}

cudaError_t launch_coeffs(spod_plan_s& p, const void* d_X, const void* d_Phi, int nmodes, int nmodes_r, int nsel,
                          const int* h_freqs, double* d_A, cudaStream_t s) {
  return p.f64 ? coeffs_t<double>(p, d_X, d_Phi, nmodes, nmodes_r, nsel, h_freqs, d_A, s)
               : coeffs_t<float>(p, d_X, d_Phi, nmodes, nmodes_r, nsel, h_freqs, d_A, s);
}

cudaError_t launch_reconstruct(spod_plan_s& p, const void* d_Phi, int nmodes, int nmodes_r, int nsel,
                               const int* h_freqs, const double* d_A, void* d_Xrec, cudaStream_t s) {
  return p.f64 ? reconstruct_t<double>(p, d_Phi, nmodes, nmodes_r, nsel, h_freqs, d_A, d_Xrec, s)
               : reconstruct_t<float>(p, d_Phi, nmodes, nmodes_r, nsel, h_freqs, d_A, d_Xrec, s);
}

}  // namespace spod
