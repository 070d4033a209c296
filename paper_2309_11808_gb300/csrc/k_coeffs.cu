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
// The two large products are plain GEMMs and go to cuBLAS (FP32 or FP64 as
// the plan); the K x K Gram of the basis, its inverse and the packing are
// kernels of this file.
#include <cublas_v2.h>

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

// B64 = B - v 1^T (B column-major K x nt, type R).
template <typename R>
__global__ void k_coeff_center(const R* __restrict__ B, const double* __restrict__ v, int K, int64_t n,
                               double* __restrict__ B64) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    B64[e] = (double)B[e] - v[e % K];
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

cudaError_t cublas_err(cublasStatus_t st) { return st == CUBLAS_STATUS_SUCCESS ? cudaSuccess : cudaErrorUnknown; }

cublasHandle_t handle_of(spod_plan_s& p, cudaStream_t s, cudaError_t* e) {
  if (!p.blas) {
    cublasHandle_t h = nullptr;
    if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) {
      *e = cudaErrorUnknown;
      return nullptr;
    }
    cublasSetMathMode(h, CUBLAS_PEDANTIC_MATH);      // FP32 stays FP32 (no TF32)
    p.blas = h;
  }
  cublasHandle_t h = static_cast<cublasHandle_t>(p.blas);
  if (cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS) *e = cudaErrorUnknown;
  return h;
}

template <typename R>
cudaError_t gemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, R alpha,
                 const R* A, int lda, const R* B, int ldb, R beta, R* C, int ldc) {
  if constexpr (sizeof(R) == 8)
    return cublas_err(cublasDgemm(h, ta, tb, m, n, k, &alpha, A, lda, B, ldb, &beta, C, ldc));
  else
    return cublas_err(cublasSgemm(h, ta, tb, m, n, k, &alpha, A, lda, B, ldb, &beta, C, ldc));
}

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
  R* B = static_cast<R*>(sc.get(sizeof(R) * (size_t)K * nt));
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
  // B = P_w X^T (column-major K x nt): X is column-major M x nt
  cublasHandle_t h = handle_of(p, s, &e);
  if (e != cudaSuccess) return e;
  e = gemm<R>(h, CUBLAS_OP_T, CUBLAS_OP_N, K, (int)nt, (int)M, (R)1, Pw, (int)M, static_cast<const R*>(d_X), (int)M,
              (R)0, B, K);
  if (e != cudaSuccess) return e;
  k_coeff_center<R><<<1024, 256, 0, s>>>(B, v, K, (int64_t)K * nt, B64);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  e = gemm<double>(h, CUBLAS_OP_N, CUBLAS_OP_N, K, (int)nt, K, 1.0, Ginv, K, B64, K, 0.0, C, K);
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
  cublasHandle_t h = handle_of(p, s, &e);
  if (e != cudaSuccess) return e;
  // X (column-major M x nt) += P_b^T C: P_b is column-major M x K
  return gemm<R>(h, CUBLAS_OP_N, CUBLAS_OP_N, (int)M, (int)nt, K, (R)1, Pb, (int)M, C, K, (R)1, X, (int)M);
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

void destroy_blas(spod_plan_s& p) {
  if (p.blas) cublasDestroy(static_cast<cublasHandle_t>(p.blas));
  p.blas = nullptr;
}

}  // namespace spod
