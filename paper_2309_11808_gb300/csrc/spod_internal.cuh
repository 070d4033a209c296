// Internal declarations shared by the translation units of libspod.so.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/spod.h"

namespace spod {

// Device-side condition bits (plan->d_flags[0]).
enum : unsigned {
  FLAG_NAN = 1u,            // non-finite Gram diagonal (non-finite input)
  FLAG_NOTCONV = 2u,        // eigen-solver hit its sweep cap
  FLAG_TIMEOUT = 4u,        // bounded device wait gave up
};

constexpr int kMaxRadixPasses = 32;
constexpr int kMaxNb = 1024;           // largest supported block count
constexpr int kEigSmemMaxNb = 48;      // eigen-solver keeps A and V in shared memory up to here

// Qhat layout of one spatial chunk.  FP32/FP64 planes are planar, element
// (f, row, m) at (f * 2 nb + row) * chunk + m.  The BF16 planes of the
// tensor-core path are blocked by kQBlock points, [chunk / kQBlock][nf][2 nb]
// [kQBlock]: the rows that one spatial tile contributes to every frequency lie
// within a few MB (a handful of pages, whatever the chunk size), and the
// K step of one frequency is a single contiguous qrows x 128-byte box for the
// tensor-core kernels.  Rows are re = l, im = nb + l for Welch block l; when
// the time mean is folded into the FFT (spod_plan_s::mean_fold) one more row,
// 2 nb, holds rho_m = sqrt(W_m) (mu_m - x_m(t = 0)) of every point (qrows =
// 2 nb + 1), the input of the rank-one mean correction of the consumers.
constexpr int kQBlock = 64;
__host__ __device__ inline int64_t qhat_blocked_offset(int nf, int qrows, int f, int row, int64_t m) {
  return (((m / kQBlock) * nf + f) * qrows + row) * kQBlock + (m % kQBlock);
}

struct FftPlan {
  int n = 0;
  int npass = 0;
  int radix[kMaxRadixPasses] = {0};
};

// Factor n into passes of radix 8, 4, 2, 3, 5.  Returns false if n has another
// prime factor.
bool make_fft_plan(int n, FftPlan* fp);

struct Workspace {
  void* base = nullptr;
  size_t bytes = 0;
};

}  // namespace spod

struct spod_plan_s {
  uint64_t uid = 0;        // unique per plan (never reused): keys cached CUDA graphs
  uint64_t version = 0;    // bumped when launch parameters change (tuning, profiling)
  spod_plan_desc desc{};
  int64_t npoints = 0, M = 0, Mpad = 0, nt = 0;
  int nvars = 0, nfft = 0, noverlap = 0, step = 0, nb = 0, nf = 0;
  double c = 0.0;        // 1 / sum(w)
  double kappa = 0.0;    // 1/nb or 1/(nb-1)
  std::vector<double> w; // window (FP64)
  std::vector<double> W; // weights (FP64)
  int device = 0;
  bool f64 = false;      // FP64 arithmetic path
  spod::FftPlan fft;

  // spatial chunking of the FFT -> Gram / modes pipeline
  int64_t chunk_points = 0;   // points per chunk (multiple of the FFT tile)
  int gram_splits = 1;        // CTAs per frequency per chunk in the Gram kernel
  int gram_splits_max = 1;    // partial-Gram slots allocated
  int gram_flush = 1;         // tensor-core Gram: 64-point blocks per tensor-memory accumulation run
  int modes_ctas = 0;         // tensor-core modes: CTAs per frequency (0 = automatic)
  int eig_max_iter = 0;       // QL iterations per eigenvalue (0 = the solver's default)
  int wait_timeout_us = 0;    // bound of every device wait, in microseconds (0 = 2 s); mirrored in d_flags[1]
  int wait_selftest = 0;      // tensor-core Gram leaves its first stage unissued (the bounded-wait self-test)
  int ring_boxr = 0;          // TMA ring FFT: rows per box (0 = ring kernel not usable)
  bool ring_ok = false;       // a TMA-fed FFT kernel (pipelined or ring) is used
  bool cplx = false;          // complex input: two-sided spectrum, complex mean
  // Views for data held in tiles (out-of-core driver): X is read as rows of
  // x_ld points starting at point x_off, Phi written as rows of phi_ld points
  // starting at point phi_off (0, 0: the full arrays, row stride M).
  int64_t x_ld = 0, x_off = 0, phi_ld = 0, phi_off = 0;
  bool pipe_ok = false;       // the pipelined kernel (compiled nfft) is used
  // The time mean folded into the pipelined FFT (real data, tensor-core
  // precisions, 2 nb + 1 rows within the 16-row MMA padding of 2 nb): the FFT
  // subtracts each column's first sample, accumulates the mean of the rest,
  // writes mu and the rho row; the Gram and the modes apply the exact rank-one
  // correction Qhat = Z - mu' What_f.  No separate mean pass reads X.
  bool mean_fold = false;
  int qrows = 0;              // Qhat rows per frequency: 2 nb (+ 1 with mean_fold)
  int pipe_tp = 16;           // its tile width in points (16 or 32; also the X map's box width)
  void* encode_fn = nullptr;  // cuTensorMapEncodeTiled
  int num_sms = 0;

  // device workspace (one allocation, carved)
  spod::Workspace ws;
  double* d_mu = nullptr;          // [M] time mean
  double* d_mupart = nullptr;      // [mean_splits][M]
  int mean_splits = 1;
  void* d_win = nullptr;           // [nfft] c * w_n, compute type
  void* d_tw = nullptr;            // [nfft] complex twiddles exp(-2 pi i k / nfft), compute type
  void* d_sqrtW = nullptr;         // [Mpad] sqrt(W) (0 in the padding), compute type
  void* d_rsqrtW = nullptr;        // [Mpad] 1/sqrt(W), compute type
  void* d_qhat = nullptr;          // [nf][2*nb][chunk_points] compute type (planar re | im); BF16 hi for tensor precisions
  void* d_qlo = nullptr;           // BF16X3: the lo part, same layout
  bool tensor = false;             // BF16 / BF16X3: Gram and modes on the tensor cores
  CUtensorMap tmap_hi;            // TMA maps of d_qhat / d_qlo: dims {chunk, 2nb, nf}, box {64, round16(2nb), 1}
  CUtensorMap tmap_lo;
  CUtensorMap tmap_hi2;           // the same planes, box {64, round16(2nb), 1, 2}: two 64-point blocks per copy
  CUtensorMap tmap_lo2;
  CUtensorMap tmap_fst_hi;         // FFT output store maps: dims {chunk, 2nb, nf}, box {16, 1, 256}
  CUtensorMap tmap_fst_lo;         //   (FP32 planes, or BF16 hi / lo)
  bool fst_maps = false;
  int fst_fbox = 0;                // frequency rows per FFT output store box
  double* d_gslot = nullptr;       // tensor path: FP64 (cta + f) slots of D = Y Y^T
  double* d_gacc = nullptr;        // tensor path: [nf][2 nb][2 nb] FP64 D accumulated over chunks
  double* d_gpart = nullptr;       // [gram_splits][nf][nb][nb][2] FP64 partial Grams
  double* d_gram = nullptr;        // [nf][nb][nb][2] reduced Gram (kappa applied)
  double* d_lam = nullptr;         // [nf][nb]
  double* d_psi = nullptr;         // [nf][nb][nb][2]
  double* d_eigws = nullptr;       // [nf][2][nbp][nbp][2] eigen-solver scratch (large nb)
  void* d_bimg = nullptr;          // tensor path: per-frequency BF16 B images of the mode GEMM
  void* d_bmat = nullptr;          // [nf][nb][nb] complex compute type: psi_k / sqrt(lambda_k / kappa), or G_f
  void* d_wc = nullptr;            // [nf] complex compute type: c sum_n w_n e^{+2 pi i f n / nfft}
  double* d_what = nullptr;        // [nf] complex FP64: What_f = c sum_n w_n e^{-2 pi i f n / nfft} (mean fold)
  void* d_radj = nullptr;          // [nf][adj_cols][radj_points] complex compute type: R_f of the adjoint, one column sub-chunk
  // spod_backward: R carries, beside its nb columns, the column Wc_f sum_l R_f[.][l]
  // (one more column of the G image) from which the kernels take the mean of
  // dL/dxt; adj_cols = nb + 1 then (not when 2 (nb + 1) exceeds the tensor-core
  // mode kernel's 128 accumulator columns: nb = 64)
  int adj_cols = 0;
  int64_t radj_points = 0;         // points per adjoint sub-chunk (a multiple of 128; 0: no adjoint, complex data)
  unsigned* d_flags = nullptr;     // [4]: [0] condition bits (cleared per fit), [1] wait bound in us

  bool fitted = false;
  bool partial = false;            // spod_fit_partial ran: the Gram of this plan's slab is in d_gram, not decomposed
  bool qhat_valid = false;         // d_qhat holds the fit's Qhat for all points (single chunk)
  cudaStream_t last_stream = nullptr;

  // staging for spod_run_host
  void* d_xstage = nullptr;
  size_t xstage_bytes = 0;
  void* d_phistage = nullptr;
  size_t phistage_bytes = 0;
  // spod_run_host(_many): second staging pair, copy streams (host to device,
  // device to host) and the events that hand buffers between the streams
  void* d_xstage2 = nullptr;
  size_t xstage2_bytes = 0;
  void* d_phistage2 = nullptr;
  size_t phistage2_bytes = 0;
  void* d_lamstage = nullptr;              // eigenvalues of each dataset of a run_host call
  size_t lamstage_bytes = 0;
  cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr;
  std::vector<cudaEvent_t> host_ev;
  double* d_gradlam = nullptr;

  // per-phase timing and launch counts
  bool prof = false;
  struct Rec { int phase; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> ev_free;
  int64_t launches[SPOD_NPHASES] = {0};
};

namespace spod {

// Launchers (each returns the first CUDA error it meets).
// Time mean of the columns [m0, m0 + mcount) of X.
cudaError_t launch_mean(const spod_plan_s& p, const void* d_X, int64_t m0, int64_t mcount, cudaStream_t s);
cudaError_t launch_fft_chunk(const spod_plan_s& p, const void* d_X, int64_t m0, int64_t mcount,
                             cudaStream_t s);
cudaError_t launch_gram_chunk(const spod_plan_s& p, int64_t mcount, bool first, cudaStream_t s);
cudaError_t launch_gram_reduce(const spod_plan_s& p, cudaStream_t s);
// Part-order sum of slab Grams [nparts][nf][nb][nb] (complex FP64) into the plan's Gram.
cudaError_t launch_gram_sum_parts(const spod_plan_s& p, const double* parts, int nparts, cudaStream_t s);
cudaError_t launch_eig(const spod_plan_s& p, cudaStream_t s);
cudaError_t launch_mode_coeffs(const spod_plan_s& p, int nmodes, cudaStream_t s);
// Modes of the points [m0, m0 + mcount) at the frequencies [f0, f1) (f1 < 0: all).
// qoff: the points' first column inside the plan's Qhat chunk; out_ld / out_off
// (when out_ld > 0): row stride and first point of the output (the adjoint's R
// sub-chunks), else the plan's Phi view.
cudaError_t launch_modes_chunk(const spod_plan_s& p, int64_t m0, int64_t mcount, int nmodes,
                               void* d_Phi, cudaStream_t s, int* nlaunch, bool adjoint = false, int f0 = 0,
                               int f1 = -1, int64_t qoff = 0, int64_t out_ld = 0, int64_t out_off = 0);
cudaError_t launch_adj_gmat(const spod_plan_s& p, const double* d_g, cudaStream_t s);
// dL/dX of the points [m0, m0 + mcount) from R held as [nf][nb][rs] starting at point roff.
cudaError_t launch_adjoint_chunk(const spod_plan_s& p, const void* d_R, int64_t rs, int64_t roff, int64_t m0,
                                 int64_t mcount, void* d_dX, cudaStream_t s);
size_t adjoint_smem_bytes(const spod_plan_s& p);

cudaError_t launch_gram_tc_chunk(const spod_plan_s& p, int64_t mcount, bool first, cudaStream_t s);
cudaError_t launch_modes_tc_chunk(const spod_plan_s& p, int64_t m0, int64_t mcount, int nmodes, void* d_Phi,
                                  cudaStream_t s, bool adjoint = false, int f0 = 0, int f1 = -1, int64_t qoff = 0,
                                  int64_t out_ld = 0, int64_t out_off = 0);
size_t gram_tc_smem_bytes(const spod_plan_s& p);
size_t modes_tc_smem_bytes(const spod_plan_s& p);
size_t modes_image_bytes(const spod_plan_s& p);
cudaError_t launch_mode_image(const spod_plan_s& p, int nmodes, cudaStream_t s);
size_t gram_simt_smem_bytes(const spod_plan_s& p);
size_t gram_tc_slot_doubles(const spod_plan_s& p, int max_ctas);
size_t gram_tc_acc_doubles(const spod_plan_s& p);
int gram_tc_ctas(const spod_plan_s& p);
cudaError_t launch_gram_tc_finish(const spod_plan_s& p, cudaStream_t s);

cudaError_t launch_eig_buffers(const double* gram, int nf, int nb, double* lam, double* psi, double* gws,
                               unsigned* flags, cudaStream_t s);

size_t fft_smem_bytes(const spod_plan_s& p);
size_t fft_ring_smem_bytes(const spod_plan_s& p);
size_t fft_ring_stage_offset(const spod_plan_s& p);
size_t fft_ring_plane_elems(const spod_plan_s& p);
bool fft_ring_usable(const spod_plan_s& p, int smem_optin);
size_t fft_pipe_smem_bytes(const spod_plan_s& p, int tp);
bool fft_pipe_usable(const spod_plan_s& p, int smem_optin);
int fft_pipe_tile(const spod_plan_s& p, int smem_optin);
cudaError_t launch_fft_pipe_chunk(const spod_plan_s& p, const CUtensorMap& xmap, const void* d_X, int64_t m0,
                                  int64_t mcount,
                                  cudaStream_t s);
cudaError_t launch_fft_ring_chunk(const spod_plan_s& p, const CUtensorMap& xmap, int64_t m0, int64_t mcount,
                                  cudaStream_t s);
size_t eig_smem_bytes(int nb);
size_t eig_tridiag_smem_bytes(int nb);
size_t eig_tridiag_gws_doubles(int nb, int nf);
cudaError_t launch_eig_tridiag(const spod_plan_s& p, cudaStream_t s);
// expansion coefficients / reconstruction (k_coeffs.cu)
int coeff_basis_size(const spod_plan_s& p, int nmodes_r, int nsel, const int* h_freqs);
cudaError_t launch_coeffs(spod_plan_s& p, const void* d_X, const void* d_Phi, int nmodes, int nmodes_r, int nsel,
                          const int* h_freqs, double* d_A, cudaStream_t s);
cudaError_t launch_reconstruct(spod_plan_s& p, const void* d_Phi, int nmodes, int nmodes_r, int nsel,
                               const int* h_freqs, const double* d_A, void* d_Xrec, cudaStream_t s);
// strided tile copy (k_tile_copy.cu)
// rows x width bytes from src (pitch spitch) to dst (pitch dpitch); bytes
// [width, dwidth) of each destination row are set to zero
cudaError_t launch_copy2d(void* dst, int64_t dpitch, const void* src, int64_t spitch, int64_t width, int64_t dwidth,
                          int64_t rows, int num_sms, cudaStream_t s);

void set_error(const std::string& msg);

}  // namespace spod
