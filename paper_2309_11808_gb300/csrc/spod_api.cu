// C ABI of libspod.so: plan validation, workspace layout and the entry points
// declared in include/spod.h.  Every step of the path runs in the kernels of
// this library; this file only validates, allocates and enqueues.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <string>

#include <cudaTypedefs.h>

#include "spod_internal.cuh"

namespace spod {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

namespace {

spod_status fail(spod_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

spod_status cuda_fail(cudaError_t e, const char* where) {
  return fail(SPOD_ECUDA, std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define SPOD_CUDA(call, where)                 \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

std::vector<double> make_window(const spod_plan_desc& d) {
  const int N = d.nfft;
  std::vector<double> w(N, 1.0);
  const double pi = 3.14159265358979323846;
  for (int n = 0; n < N; ++n) {
    switch (d.window) {
      case SPOD_WIN_HAMMING: w[n] = N > 1 ? 0.54 - 0.46 * std::cos(2.0 * pi * n / (N - 1)) : 1.0; break;
      case SPOD_WIN_HAMMING_PERIODIC: w[n] = 0.54 - 0.46 * std::cos(2.0 * pi * n / N); break;
      case SPOD_WIN_HANN: w[n] = N > 1 ? 0.5 - 0.5 * std::cos(2.0 * pi * n / (N - 1)) : 1.0; break;
      case SPOD_WIN_RECT: w[n] = 1.0; break;
      case SPOD_WIN_USER: w[n] = d.user_window[n]; break;
    }
  }
  return w;
}

size_t elem_bytes(spod_dtype t) {
  switch (t) {
    case SPOD_F64: return 8;
    case SPOD_F32: return 4;
    case SPOD_BF16: return 2;
    case SPOD_C64: return 8;
    default: return 16;
  }
}
bool is_complex(spod_dtype t) { return t == SPOD_C64 || t == SPOD_C128; }

spod_status check_plan(spod_plan_t p) {
  if (!p) return fail(SPOD_EINVAL, "plan is NULL");
  return SPOD_OK;
}

spod_status read_flags(spod_plan_t p) {
  unsigned h[4] = {0, 0, 0, 0};
  SPOD_CUDA(cudaMemcpy(h, p->d_flags, sizeof(h), cudaMemcpyDeviceToHost), "read device flags");
  if (h[0] & FLAG_TIMEOUT) return fail(SPOD_ETIMEOUT, "a bounded device wait gave up");
  if (h[0] & FLAG_NAN) return fail(SPOD_ENANINPUT, "non-finite values in X (Gram diagonal not finite)");
  if (h[0] & FLAG_NOTCONV) return fail(SPOD_ENOTCONVERGED, "eigen-solver reached its sweep cap");
  return SPOD_OK;
}

cudaEvent_t take_event(spod_plan_s* p) {
  if (!p->ev_free.empty()) {
    cudaEvent_t e = p->ev_free.back();
    p->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Bracket one phase of a call with events on its stream (when profiling).
struct Phase {
  spod_plan_s* p;
  int ph;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  int n;
  Phase(spod_plan_s* p_, int ph_, cudaStream_t s_, int nlaunch) : p(p_), ph(ph_), s(s_), n(nlaunch) {
    if (p->prof) {
      a = take_event(p);
      if (a) cudaEventRecord(a, s);
    }
  }
  ~Phase() {
    p->launches[ph] += n;
    if (a) {
      cudaEvent_t b = take_event(p);
      if (b) {
        cudaEventRecord(b, s);
        p->recs.push_back({ph, a, b});
      } else {
        p->ev_free.push_back(a);
      }
    }
  }
};

void* driver_encode_fn() {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess) return nullptr;
  return fn;
}

// TMA map of X for the ring FFTs: dims {M, nt}, box {tile points, ring_boxr rows}.
spod_status make_x_map(const spod_plan_s* p, const void* d_X, CUtensorMap* map) {
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p->encode_fn);
  if (!encode) return fail(SPOD_ECUDA, "cuTensorMapEncodeTiled not available");
  // complex data: a [nt][2M] array of interleaved real components
  const spod_dtype t = p->desc.in_dtype;
  const int64_t xld = p->x_ld ? p->x_ld : p->M;     // tiled data: the tile's width
  const int64_t cols = p->cplx ? 2 * xld : xld;
  const size_t el = p->cplx ? elem_bytes(t) / 2 : elem_bytes(t);
  const CUtensorMapDataType dt = t == SPOD_F64 || t == SPOD_C128 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                 : t == SPOD_F32 || t == SPOD_C64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                                  : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)p->nt};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * el};
  const cuuint32_t box[2] = {(cuuint32_t)(p->pipe_ok ? p->pipe_tp : 16), (cuuint32_t)p->ring_boxr};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(map, dt, 2, const_cast<void*>(d_X), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(SPOD_ECUDA, "cuTensorMapEncodeTiled (X) failed (" + std::to_string((int)r) + ")");
  return SPOD_OK;
}

// FFT of one spatial chunk: the TMA-ring kernel when the shape allows it.
spod_status run_fft_chunk(spod_plan_s* p, const void* d_X, const CUtensorMap* xmap, int64_t m0, int64_t mc,
                          cudaStream_t s) {
  // the folded mean lives in the pipelined kernel only (mean_fold implies pipe_ok,
  // and every caller builds the X map when ring_ok holds)
  if (p->mean_fold && !xmap) return fail(SPOD_EUNSUPPORTED, "folded time mean without the X tensor map");
  cudaError_t e = !xmap        ? launch_fft_chunk(*p, d_X, m0, mc, s)
                  : p->pipe_ok ? launch_fft_pipe_chunk(*p, *xmap, d_X, m0, mc, s)
                               : launch_fft_ring_chunk(*p, *xmap, m0, mc, s);
  if (e != cudaSuccess) return cuda_fail(e, "fft kernel");
  return SPOD_OK;
}

// TMA store maps for the FFT output planes: boxes of 16 points x 1 row x fst_fbox frequencies.
void make_fft_store_maps(spod_plan_s* p) {
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p->encode_fn);
  if (!encode || p->f64) return;
  const size_t el = p->tensor ? 2 : 4;
  const CUtensorMapDataType dt = p->tensor ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const int nbox = (p->nf + 255) / 256;
  // <= 256 rows per box, a multiple of 4 so every box starts 128-byte aligned in shared memory
  p->fst_fbox = ((p->nf + nbox - 1) / nbox + 3) / 4 * 4;
  // FP32: planar {chunk, 2 nb, nf}; BF16: blocked {64, 2 nb, nf, chunk / 64} (qhat_blocked_offset)
  const int rank = p->tensor ? 4 : 3;
  cuuint64_t dims[4], strides[3];
  if (p->tensor) {
    dims[0] = kQBlock; dims[1] = p->qrows; dims[2] = p->nf; dims[3] = p->chunk_points / kQBlock;
    strides[0] = (cuuint64_t)kQBlock * el;
    strides[1] = strides[0] * p->qrows;
    strides[2] = strides[1] * p->nf;
  } else {
    dims[0] = p->chunk_points; dims[1] = 2 * p->nb; dims[2] = p->nf;
    strides[0] = (cuuint64_t)p->chunk_points * el;
    strides[1] = strides[0] * 2 * p->nb;
  }
  const cuuint32_t box[4] = {16, 1, (cuuint32_t)p->fst_fbox, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  void* bases[2] = {p->d_qhat, p->d_qlo ? p->d_qlo : p->d_qhat};
  CUtensorMap* maps[2] = {&p->tmap_fst_hi, &p->tmap_fst_lo};
  for (int i = 0; i < 2; ++i) {
    CUresult r = encode(maps[i], dt, rank, bases[i], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return;   // the ring FFT is then not used
  }
  p->fst_maps = true;
}

// TMA maps of the BF16 Qhat planes: dims {64 points, 2 nb rows, nf, chunk / 64},
// box {64 points, 2 nb rounded up to 16 rows, 1, 1}; 128-byte swizzle.
spod_status make_qhat_maps(spod_plan_s* p) {
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p->encode_fn);
  if (!encode) return fail(SPOD_ECUDA, "cuTensorMapEncodeTiled not available from the driver");
  // blocked layout [chunk / 64][nf][2 nb][64] (qhat_blocked_offset): one box =
  // one frequency's rows over one 64-point K step; rows past 2 nb read as zero
  const cuuint64_t dims[4] = {(cuuint64_t)kQBlock, (cuuint64_t)p->qrows, (cuuint64_t)p->nf,
                              (cuuint64_t)(p->chunk_points / kQBlock)};
  const cuuint64_t row = (cuuint64_t)kQBlock * 2;
  const cuuint64_t strides[3] = {row, row * p->qrows, row * p->qrows * p->nf};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  void* bases[2] = {p->d_qhat, p->d_qlo ? p->d_qlo : p->d_qhat};
  CUtensorMap* maps[4] = {&p->tmap_hi, &p->tmap_lo, &p->tmap_hi2, &p->tmap_lo2};
  for (int i = 0; i < 4; ++i) {
    // boxes of one 64-point block, and of two consecutive blocks (fewer, larger copies)
    const cuuint32_t box[4] = {(cuuint32_t)kQBlock, (cuuint32_t)((2 * p->nb + 15) / 16 * 16), 1, i < 2 ? 1u : 2u};
    CUresult r = encode(maps[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, bases[i & 1], dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SPOD_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  }
  return SPOD_OK;
}

}  // namespace
}  // namespace spod

using namespace spod;

extern "C" {

const char* spod_last_error(void) { return g_err.c_str(); }

const char* spod_version(void) { return "spod-gb300 0.1 (sm_103a)"; }

spod_status spod_desc_init(spod_plan_desc* d) {
  if (!d) return fail(SPOD_EINVAL, "desc is NULL");
  std::memset(d, 0, sizeof(*d));
  d->ndim = 1;
  d->dims[0] = 1;
  d->dims[1] = 1;
  d->dims[2] = 1;
  d->nvars = 1;
  d->window = SPOD_WIN_HAMMING;
  d->dt = 1.0;
  d->in_dtype = SPOD_F32;
  d->precision = SPOD_PREC_FP32;
  d->norm = SPOD_NORM_NB;
  d->subtract_mean = 1;
  d->chunk_points = 0;
  d->mean_in_fft = 1;
  return SPOD_OK;
}

static std::atomic<uint64_t> g_plan_uid{0};

spod_status spod_plan_create(const spod_plan_desc* d, spod_plan_t* out) {
  if (!out) return fail(SPOD_EINVAL, "out is NULL");
  *out = nullptr;
  if (!d) return fail(SPOD_EINVAL, "desc is NULL");
  if (d->ndim < 1 || d->ndim > 3) return fail(SPOD_EINVAL, "ndim must be 1..3");
  int64_t npoints = 1;
  for (int i = 0; i < d->ndim; ++i) {
    if (d->dims[i] <= 0) return fail(SPOD_EINVAL, "dims must be positive");
    if (npoints > (int64_t(1) << 40) / d->dims[i]) return fail(SPOD_EINVAL, "grid too large");
    npoints *= d->dims[i];
  }
  if (d->nvars < 1) return fail(SPOD_EINVAL, "nvars must be >= 1");
  const int64_t M = npoints * d->nvars;
  if (d->nfft < 2) return fail(SPOD_EINVAL, "nfft must be >= 2");
  if (d->noverlap < 0 || d->noverlap >= d->nfft) return fail(SPOD_EINVAL, "need 0 <= noverlap < nfft");
  if (d->nt < d->nfft) return fail(SPOD_EINVAL, "need nfft <= nt");
  if (d->in_dtype != SPOD_F64 && d->in_dtype != SPOD_F32 && d->in_dtype != SPOD_BF16 && d->in_dtype != SPOD_C64 &&
      d->in_dtype != SPOD_C128)
    return fail(SPOD_EINVAL, "unknown in_dtype");
  if (d->precision < SPOD_PREC_FP64 || d->precision > SPOD_PREC_BF16X3) return fail(SPOD_EINVAL, "unknown precision");
  if (d->norm != SPOD_NORM_NB && d->norm != SPOD_NORM_NB_MINUS_1) return fail(SPOD_EINVAL, "unknown norm");
  if (d->window < SPOD_WIN_HAMMING || d->window > SPOD_WIN_USER) return fail(SPOD_EINVAL, "unknown window");
  if (d->window == SPOD_WIN_USER && !d->user_window) return fail(SPOD_EINVAL, "user_window is NULL");
  if (!(d->dt > 0.0) || !std::isfinite(d->dt)) return fail(SPOD_EINVAL, "dt must be positive and finite");
  if (d->chunk_points < 0) return fail(SPOD_EINVAL, "chunk_points must be >= 0");

  spod_plan_s* p = new (std::nothrow) spod_plan_s();
  if (!p) return fail(SPOD_ENOMEM, "host allocation failed");
  p->desc = *d;
  p->uid = ++g_plan_uid;
  p->desc.user_window = nullptr;
  p->desc.weights = nullptr;
  p->npoints = npoints;
  p->M = M;
  p->nvars = d->nvars;
  p->nt = d->nt;
  p->nfft = d->nfft;
  p->noverlap = d->noverlap;
  p->step = d->nfft - d->noverlap;
  p->nb = (int)((d->nt - d->noverlap) / p->step);
  p->cplx = is_complex(d->in_dtype);
  p->nf = p->cplx ? d->nfft : d->nfft / 2 + 1;     // two-sided for complex data
  p->f64 = d->precision == SPOD_PREC_FP64;
  p->tensor = d->precision == SPOD_PREC_BF16 || d->precision == SPOD_PREC_BF16X3;
  auto bail = [&](spod_status st, const std::string& m) {
    spod_plan_destroy(p);
    return fail(st, m);
  };
  if (p->nb < 1) return bail(SPOD_EINVAL, "no complete block");
  if (d->norm == SPOD_NORM_NB_MINUS_1 && p->nb < 2) return bail(SPOD_EINVAL, "nb-1 normalisation needs nb >= 2");
  if (p->nb > 256) return bail(SPOD_EUNSUPPORTED, "nb > 256 blocks is not supported");
  if (!make_fft_plan(d->nfft, &p->fft)) return bail(SPOD_EUNSUPPORTED, "nfft must factor into 2, 3 and 5");
  if (d->nfft > 1024) return bail(SPOD_EUNSUPPORTED, "nfft > 1024 is not supported by the block FFT kernel");
  if (p->tensor && p->nb > 64)
    return bail(SPOD_EUNSUPPORTED, "BF16 / BF16X3 precisions support nb <= 64 (2 nb rows per MMA tile)");
  p->adj_cols = p->nb + ((!p->tensor || 2 * (p->nb + 1) <= 128) ? 1 : 0);
  p->kappa = 1.0 / (d->norm == SPOD_NORM_NB ? (double)p->nb : (double)(p->nb - 1));

  p->w = make_window(*d);
  double sw = 0.0;
  for (double v : p->w) {
    if (!std::isfinite(v)) return bail(SPOD_EINVAL, "window has non-finite entries");
    sw += v;
  }
  if (!(std::fabs(sw) > 0.0)) return bail(SPOD_EINVAL, "window sums to zero");
  p->c = 1.0 / sw;
  p->W.assign(M, 1.0);
  if (d->weights) {
    for (int64_t m = 0; m < M; ++m) {
      const double v = d->weights[m];
      if (!(v > 0.0) || !std::isfinite(v)) return bail(SPOD_EINVAL, "weights must be positive and finite");
      p->W[m] = v;
    }
  }

  if (cudaGetDevice(&p->device) != cudaSuccess) return bail(SPOD_ECUDA, "no CUDA device");
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, p->device) != cudaSuccess) return bail(SPOD_ECUDA, "device query failed");
  p->num_sms = prop.multiProcessorCount;
  p->encode_fn = driver_encode_fn();
  {
    // ring FFT: TMA boxes of ring_boxr rows must tile both nfft and step (largest such <= 256)
    int g = p->nfft, b = p->step;
    while (b) { const int t = g % b; g = b; b = t; }
    int boxr = 0;
    for (int dv = std::min(g, 256); dv >= 1; --dv)
      if (g % dv == 0) { boxr = dv; break; }
    const size_t rowb = 16 * (is_complex(d->in_dtype) ? elem_bytes(d->in_dtype) / 2 : elem_bytes(d->in_dtype));
    p->ring_boxr = ((size_t)boxr * rowb) % 128 == 0 ? boxr : 0;
  }
  if (fft_smem_bytes(*p) > (size_t)prop.sharedMemPerBlockOptin)
    return bail(SPOD_EUNSUPPORTED, "nfft too large for the shared-memory FFT");
  if (!p->tensor && gram_simt_smem_bytes(*p) > (size_t)prop.sharedMemPerBlockOptin)
    return bail(SPOD_EUNSUPPORTED, "nb too large for the shared-memory Gram kernel");
  if (p->tensor && (gram_tc_smem_bytes(*p) > (size_t)prop.sharedMemPerBlockOptin ||
                    modes_tc_smem_bytes(*p) > (size_t)prop.sharedMemPerBlockOptin))
    return bail(SPOD_EUNSUPPORTED, "tensor-core kernels do not fit in shared memory for this nb");
  if (p->tensor && prop.major < 10) return bail(SPOD_EUNSUPPORTED, "tensor-core path needs an sm_100-class GPU");

  // ---- which FFT kernel; whether the time mean is folded into it
  {
    const bool q = p->encode_fn != nullptr;
    if (q) p->pipe_tp = fft_pipe_tile(*p, (int)prop.sharedMemPerBlockOptin);
    p->pipe_ok = q && fft_pipe_usable(*p, (int)prop.sharedMemPerBlockOptin);
  }
  p->mean_fold = d->mean_in_fft && p->tensor && p->pipe_ok && !p->cplx && d->subtract_mean &&
                 (2 * p->nb + 1 + 15) / 16 == (2 * p->nb + 15) / 16;
  p->qrows = 2 * p->nb + (p->mean_fold ? 1 : 0);

  // ---- sizes of the workspace
  const size_t R = p->f64 ? 8 : 4;
  const int64_t tile = 64;
  // Qhat bytes per point: FP64/FP32 planar, or BF16 hi (+ lo for BF16X3)
  const size_t qelem = p->tensor ? 2 : R;
  const size_t nq = d->precision == SPOD_PREC_BF16X3 ? 2 : 1;
  const size_t per_point = (size_t)p->nf * p->qrows * qelem * nq;
  int64_t chunk = d->chunk_points;
  if (chunk == 0) {
    // whole-array Qhat up to the larger of 40 GiB and 35 % of the device memory
    // free now (the modes then reuse it), else spatial chunks
    size_t budget = (size_t)40 << 30, free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) budget = std::max(budget, free_b / 100 * 35);
    else cudaGetLastError();
    chunk = (int64_t)std::min<size_t>((size_t)M, std::max<size_t>(budget / per_point, tile));
  }
  chunk = std::min<int64_t>(chunk, M);
  chunk = ((chunk + tile - 1) / tile) * tile;
  p->chunk_points = chunk;
  p->Mpad = ((M + tile - 1) / tile) * tile;
  {
    const int64_t ctas = ((p->cplx ? 2 * M : M) + 255) / 256;
    int64_t sp = (1216 + ctas - 1) / ctas;
    sp = std::max<int64_t>(1, std::min<int64_t>(sp, p->nt / 16 > 0 ? p->nt / 16 : 1));
    p->mean_splits = (int)std::min<int64_t>(sp, 4096);
  }
  if (p->tensor) {
    // persistent tensor-core Gram: one CTA per SM by default (tunable up to two per SM)
    p->gram_splits = p->num_sms > 0 ? p->num_sms : 148;
    p->gram_splits_max = 2 * p->gram_splits;
  } else {
    int64_t s = (2048 + p->nf - 1) / p->nf;
    s = std::max<int64_t>(1, std::min<int64_t>(s, (chunk + 255) / 256));
    p->gram_splits = (int)s;
    p->gram_splits_max = (int)std::max<int64_t>(s, std::min<int64_t>(32, (chunk + 255) / 256));
  }
  const int nb = p->nb, nf = p->nf;
  size_t off = 0;
  auto carve = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  const size_t o_flags = carve(4 * sizeof(unsigned));
  const int64_t Mr = p->cplx ? 2 * M : M;          // real columns of X (complex: re, im interleaved)
  const size_t o_mu = carve(sizeof(double) * Mr);
  const size_t o_mupart = carve(sizeof(double) * Mr * p->mean_splits);
  const size_t o_win = carve(R * p->nfft);
  const size_t o_tw = carve(2 * R * p->nfft);
  const size_t o_sqrtW = carve(R * p->Mpad);
  const size_t o_rsqrtW = carve(R * p->Mpad);
  const size_t o_gpart = p->tensor ? 0 : carve(sizeof(double) * 2 * (size_t)p->gram_splits_max * nf * nb * nb);
  const size_t o_gslot = p->tensor ? carve(sizeof(double) * gram_tc_slot_doubles(*p, p->gram_splits_max)) : 0;
  const size_t o_gacc = p->tensor ? carve(sizeof(double) * gram_tc_acc_doubles(*p)) : 0;
  const size_t o_gram = carve(sizeof(double) * 2 * (size_t)nf * nb * nb);
  const size_t o_lam = carve(sizeof(double) * (size_t)nf * nb);
  const size_t o_psi = carve(sizeof(double) * 2 * (size_t)nf * nb * nb);
  const size_t o_eigws = nb > kEigSmemMaxNb ? carve(sizeof(double) * eig_tridiag_gws_doubles(nb, nf)) : 0;
  const size_t o_bmat = carve(2 * R * (size_t)nf * nb * p->adj_cols);
  const size_t o_bimg = p->tensor ? carve(modes_image_bytes(*p)) : 0;
  const size_t o_wc = carve(2 * R * (size_t)nf);
  const size_t o_what = carve(2 * sizeof(double) * (size_t)nf);
  // R_f of the adjoint, one column sub-chunk at a time: at most 2 GiB (real data only),
  // enough columns for several waves of the adjoint kernel's 16-point CTAs
  if (!p->cplx) {
    const size_t rpp = 2 * R * (size_t)nf * p->adj_cols;
    const int64_t want = std::max<int64_t>(128, (int64_t)(((size_t)2 << 30) / rpp) / 128 * 128);
    p->radj_points = std::min<int64_t>((chunk + 127) / 128 * 128, want);
  }
  const size_t o_radj = p->radj_points ? carve(2 * R * (size_t)nf * p->adj_cols * (size_t)p->radj_points) : 0;
  const size_t o_qhat = carve(per_point * (size_t)chunk);
  p->ws.bytes = off;
  {
    DeviceGuard g(p->device);
    cudaError_t e = cudaMalloc(&p->ws.base, p->ws.bytes);
    if (e != cudaSuccess) {
      p->ws.base = nullptr;
      cudaGetLastError();
      return bail(SPOD_ENOMEM, "device workspace allocation failed (" + std::to_string(p->ws.bytes) + " bytes)");
    }
  }
  char* b = static_cast<char*>(p->ws.base);
  p->d_flags = reinterpret_cast<unsigned*>(b + o_flags);
  p->d_mu = reinterpret_cast<double*>(b + o_mu);
  p->d_mupart = reinterpret_cast<double*>(b + o_mupart);
  p->d_win = b + o_win;
  p->d_tw = b + o_tw;
  p->d_sqrtW = b + o_sqrtW;
  p->d_rsqrtW = b + o_rsqrtW;
  if (p->tensor) {
    p->d_gslot = reinterpret_cast<double*>(b + o_gslot);
    p->d_gacc = reinterpret_cast<double*>(b + o_gacc);
  } else {
    p->d_gpart = reinterpret_cast<double*>(b + o_gpart);
  }
  p->d_gram = reinterpret_cast<double*>(b + o_gram);
  p->d_lam = reinterpret_cast<double*>(b + o_lam);
  p->d_psi = reinterpret_cast<double*>(b + o_psi);
  p->d_eigws = nb > kEigSmemMaxNb ? reinterpret_cast<double*>(b + o_eigws) : nullptr;
  p->d_bmat = b + o_bmat;
  if (p->tensor) p->d_bimg = b + o_bimg;
  p->d_wc = b + o_wc;
  p->d_what = reinterpret_cast<double*>(b + o_what);
  if (p->radj_points) p->d_radj = b + o_radj;
  p->d_qhat = b + o_qhat;
  if (d->precision == SPOD_PREC_BF16X3)
    p->d_qlo = b + o_qhat + (size_t)p->nf * p->qrows * 2 * (size_t)chunk;
  make_fft_store_maps(p);
  // the runtime-radix ring kernel (real data only, needs the store maps); complex
  // data takes the pipelined kernel (compiled nfft) or the per-block one
  p->ring_ok = p->pipe_ok || (!p->cplx && p->encode_fn &&
                              fft_ring_usable(*p, (int)prop.sharedMemPerBlockOptin));
  if (p->tensor) {
    if (spod_status st = make_qhat_maps(p)) {
      std::string msg = spod_last_error();
      spod_plan_destroy(p);
      return fail(st, msg);
    }
  }

  // ---- constant tables (host FP64, rounded once to the compute type)
  {
    const int N = p->nfft;
    std::vector<double> win(N), tw(2 * N), wc(2 * (size_t)p->nf, 0.0);
    const double pi = 3.14159265358979323846;
    for (int n = 0; n < N; ++n) {
      win[n] = p->c * p->w[n];
      const double ang = 2.0 * pi * (double)n / (double)N;   // n < N: already reduced
      tw[2 * n] = std::cos(ang);
      tw[2 * n + 1] = -std::sin(ang);
    }
    std::vector<double> sq(p->Mpad, 0.0), rsq(p->Mpad, 0.0);
    for (int64_t m = 0; m < M; ++m) {
      sq[m] = std::sqrt(p->W[m]);
      rsq[m] = 1.0 / sq[m];
    }
    DeviceGuard g(p->device);
    auto up = [&](void* dst, const std::vector<double>& v) -> cudaError_t {
      if (p->f64) return cudaMemcpy(dst, v.data(), v.size() * 8, cudaMemcpyHostToDevice);
      std::vector<float> f(v.begin(), v.end());
      return cudaMemcpy(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice);
    };
    cudaError_t e = up(p->d_win, win);
    if (e == cudaSuccess) e = up(p->d_tw, tw);
    if (e == cudaSuccess) e = up(p->d_sqrtW, sq);
    if (e == cudaSuccess) e = up(p->d_rsqrtW, rsq);
    if (e == cudaSuccess) {
      // Wc_f = c sum_n w_n exp(+2 pi i f n / N), angle reduced exactly in integers
      for (int f = 0; f < p->nf; ++f) {
        double re = 0.0, im = 0.0;
        for (int n = 0; n < N; ++n) {
          const double ang = 2.0 * pi * (double)(((int64_t)f * n) % N) / (double)N;
          re += p->w[n] * std::cos(ang);
          im += p->w[n] * std::sin(ang);
        }
        wc[2 * f] = p->c * re;
        wc[2 * f + 1] = p->c * im;
      }
      e = up(p->d_wc, wc);
      if (e == cudaSuccess) {
        // What_f = c sum_n w_n exp(-2 pi i f n / N) = conj(Wc_f): the DFT of
        // the device window (c w_n) at the scale of the stored Qhat, in FP64,
        // for the rank-one correction of the folded mean
        std::vector<double> wh(2 * (size_t)p->nf);
        for (int f = 0; f < p->nf; ++f) {
          double re = 0.0, im = 0.0;
          for (int n = 0; n < N; ++n) {
            const double ang = 2.0 * pi * (double)(((int64_t)f * n) % N) / (double)N;
            re += p->w[n] * std::cos(ang);
            im -= p->w[n] * std::sin(ang);
          }
          wh[2 * f] = p->c * re;
          wh[2 * f + 1] = p->c * im;
        }
        e = cudaMemcpy(p->d_what, wh.data(), wh.size() * sizeof(double), cudaMemcpyHostToDevice);
      }
    }
    if (e == cudaSuccess) e = cudaMemset(p->d_flags, 0, 4 * sizeof(unsigned));
    if (e != cudaSuccess) {
      spod_status st = cuda_fail(e, "upload tables");
      spod_plan_destroy(p);
      return st;
    }
  }
  *out = p;
  return SPOD_OK;
}

spod_status spod_plan_destroy(spod_plan_t p) {
  if (!p) return SPOD_OK;
  {
    DeviceGuard g(p->device);
    if (p->ws.base) {
      cudaDeviceSynchronize();
      cudaFree(p->ws.base);
    }
    if (p->d_xstage) cudaFree(p->d_xstage);
    if (p->d_phistage) cudaFree(p->d_phistage);
    if (p->d_gradlam) cudaFree(p->d_gradlam);
    for (auto& r : p->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : p->ev_free) cudaEventDestroy(e);
    if (p->d_xstage2) cudaFree(p->d_xstage2);
    if (p->d_lamstage) cudaFree(p->d_lamstage);
    if (p->d_phistage2) cudaFree(p->d_phistage2);
    for (auto e : p->host_ev) cudaEventDestroy(e);
    if (p->h2d_stream) cudaStreamDestroy(p->h2d_stream);
    if (p->d2h_stream) cudaStreamDestroy(p->d2h_stream);
  }
  delete p;
  return SPOD_OK;
}

spod_status spod_plan_get_info(spod_plan_t p, spod_plan_info* info) {
  if (spod_status st = check_plan(p)) return st;
  if (!info) return fail(SPOD_EINVAL, "info is NULL");
  info->M = p->M;
  info->nt = p->nt;
  info->nfft = p->nfft;
  info->noverlap = p->noverlap;
  info->step = p->step;
  info->nb = p->nb;
  info->nf = p->nf;
  info->device = p->device;
  info->workspace_bytes = p->ws.bytes;
  info->chunk_points = p->chunk_points;
  info->mean_in_fft = p->mean_fold ? 1 : 0;
  return SPOD_OK;
}

static spod_status check_ptr(const void* ptr, const char* what) {
  if (!ptr) return fail(SPOD_EINVAL, std::string(what) + " is NULL");
  if (reinterpret_cast<uintptr_t>(ptr) % 16 != 0) return fail(SPOD_EINVAL, std::string(what) + " must be 16-byte aligned");
  return SPOD_OK;
}

// The fit over spatial chunks of at most w points (w <= chunk_points): per
// chunk the time mean of its columns, the FFT into Qhat and the Gram partial
// sums; then the reduction and the eigen-solve.
static spod_status fit_impl(spod_plan_t p, const void* d_X, cudaStream_t s, int64_t w, bool eig = true) {
  p->fitted = false;
  p->partial = false;
  p->qhat_valid = false;
  SPOD_CUDA(cudaMemsetAsync(p->d_flags, 0, sizeof(unsigned), s), "clear flags");   // [1] is the wait bound
  if (!p->desc.subtract_mean)
    SPOD_CUDA(cudaMemsetAsync(p->d_mu, 0, sizeof(double) * p->M * (p->cplx ? 2 : 1), s), "zero mean");
  alignas(64) CUtensorMap xmap;
  const CUtensorMap* xm = nullptr;
  if (p->ring_ok) {
    if (spod_status st = make_x_map(p, d_X, &xmap)) return st;
    xm = &xmap;
  }
  int64_t nchunks = 0;
  for (int64_t m0 = 0; m0 < p->M; m0 += w, ++nchunks) {
    const int64_t mc = std::min<int64_t>(w, p->M - m0);
    if (p->desc.subtract_mean && !p->mean_fold) {
      Phase ph(p, SPOD_PHASE_MEAN, s, 2);
      SPOD_CUDA(launch_mean(*p, d_X, m0, mc, s), "mean kernel");
    }
    {
      Phase ph(p, SPOD_PHASE_FFT, s, 1);
      if (spod_status st = run_fft_chunk(p, d_X, xm, m0, mc, s)) return st;
    }
    Phase ph(p, SPOD_PHASE_GRAM, s, p->tensor ? 2 : 1);
    if (p->tensor) SPOD_CUDA(launch_gram_tc_chunk(*p, mc, m0 == 0, s), "tensor-core gram kernel");
    else SPOD_CUDA(launch_gram_chunk(*p, mc, m0 == 0, s), "gram kernel");
  }
  {
    Phase ph(p, SPOD_PHASE_REDUCE, s, 1);
    if (p->tensor) SPOD_CUDA(launch_gram_tc_finish(*p, s), "gram finish kernel");
    else SPOD_CUDA(launch_gram_reduce(*p, s), "gram reduce kernel");
  }
  if (eig) {
    Phase ph(p, SPOD_PHASE_EIG, s, 1);
    SPOD_CUDA(launch_eig_tridiag(*p, s), "eigen-solver kernel");
  }
  p->fitted = eig;
  p->partial = !eig;
  p->qhat_valid = nchunks == 1;
  p->last_stream = s;
  return SPOD_OK;
}

spod_status spod_fit(spod_plan_t p, const void* d_X, void* stream) {
  if (spod_status st = check_plan(p)) return st;
  if (spod_status st = check_ptr(d_X, "d_X")) return st;
  DeviceGuard g(p->device);
  if (!g.ok) return fail(SPOD_ECUDA, "cannot select the plan's device");
  return fit_impl(p, d_X, static_cast<cudaStream_t>(stream), p->chunk_points);
}

spod_status spod_fit_partial(spod_plan_t p, const void* d_X, double* d_gram, void* stream) {
  if (spod_status st = check_plan(p)) return st;
  if (spod_status st = check_ptr(d_X, "d_X")) return st;
  if (spod_status st = check_ptr(d_gram, "d_gram")) return st;
  DeviceGuard g(p->device);
  if (!g.ok) return fail(SPOD_ECUDA, "cannot select the plan's device");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (spod_status st = fit_impl(p, d_X, s, p->chunk_points, false)) return st;
  const size_t gb = 2 * sizeof(double) * (size_t)p->nf * p->nb * p->nb;
  SPOD_CUDA(cudaMemcpyAsync(d_gram, p->d_gram, gb, cudaMemcpyDeviceToDevice, s), "copy the slab Gram");
  return SPOD_OK;
}

spod_status spod_fit_from_grams(spod_plan_t p, const double* d_grams, int nparts, void* stream) {
  if (spod_status st = check_plan(p)) return st;
  if (!p->partial) return fail(SPOD_ESTATE, "spod_fit_from_grams before spod_fit_partial on this plan");
  if (nparts < 1) return fail(SPOD_EINVAL, "nparts must be >= 1");
  if (spod_status st = check_ptr(d_grams, "d_grams")) return st;
  DeviceGuard g(p->device);
  if (!g.ok) return fail(SPOD_ECUDA, "cannot select the plan's device");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  {
    Phase ph(p, SPOD_PHASE_REDUCE, s, 1);
    SPOD_CUDA(launch_gram_sum_parts(*p, d_grams, nparts, s), "slab Gram sum kernel");
  }
  {
    Phase ph(p, SPOD_PHASE_EIG, s, 1);
    SPOD_CUDA(launch_eig_tridiag(*p, s), "eigen-solver kernel");
  }
  p->fitted = true;
  p->last_stream = s;
  return SPOD_OK;
}

spod_status spod_sync(spod_plan_t p, void* stream) {
  if (spod_status st = check_plan(p)) return st;
  DeviceGuard g(p->device);
  SPOD_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "stream synchronize");
  return read_flags(p);
}

spod_status spod_get_eigs(spod_plan_t p, double* lambda, double* psi, int on_device) {
  if (spod_status st = check_plan(p)) return st;
  if (!p->fitted) return fail(SPOD_ESTATE, "spod_get_eigs before spod_fit");
  if (!lambda) return fail(SPOD_EINVAL, "lambda is NULL");
  DeviceGuard g(p->device);
  const size_t nl = sizeof(double) * (size_t)p->nf * p->nb;
  const size_t npsi = 2 * sizeof(double) * (size_t)p->nf * p->nb * p->nb;
  if (on_device) {
    SPOD_CUDA(cudaMemcpyAsync(lambda, p->d_lam, nl, cudaMemcpyDeviceToDevice, p->last_stream), "copy lambda");
    if (psi) SPOD_CUDA(cudaMemcpyAsync(psi, p->d_psi, npsi, cudaMemcpyDeviceToDevice, p->last_stream), "copy psi");
    return SPOD_OK;
  }
  SPOD_CUDA(cudaStreamSynchronize(p->last_stream), "stream synchronize");
  SPOD_CUDA(cudaMemcpy(lambda, p->d_lam, nl, cudaMemcpyDeviceToHost), "copy lambda");
  if (psi) SPOD_CUDA(cudaMemcpy(psi, p->d_psi, npsi, cudaMemcpyDeviceToHost), "copy psi");
  return read_flags(p);
}

spod_status spod_get_gram(spod_plan_t p, double* gram) {
  if (spod_status st = check_plan(p)) return st;
  if (!p->fitted) return fail(SPOD_ESTATE, "spod_get_gram before spod_fit");
  if (!gram) return fail(SPOD_EINVAL, "gram is NULL");
  DeviceGuard g(p->device);
  SPOD_CUDA(cudaStreamSynchronize(p->last_stream), "stream synchronize");
  SPOD_CUDA(cudaMemcpy(gram, p->d_gram, 2 * sizeof(double) * (size_t)p->nf * p->nb * p->nb, cudaMemcpyDeviceToHost),
            "copy gram");
  return SPOD_OK;
}

spod_status spod_get_freqs(spod_plan_t p, double* freqs) {
  if (spod_status st = check_plan(p)) return st;
  if (!freqs) return fail(SPOD_EINVAL, "freqs is NULL");
  for (int f = 0; f < p->nf; ++f) {
    const int fs = (p->cplx && f >= (p->nfft + 1) / 2) ? f - p->nfft : f;
    freqs[f] = (double)fs / ((double)p->nfft * p->desc.dt);
  }
  return SPOD_OK;
}

// The modes: over spatial chunks of the plan (Qhat recomputed per chunk)
// unless the fit left all of Qhat in place; then, with nrange > 0, over
// nrange frequency ranges, recording done[r] after range r (Phi is
// frequency-major, so a range is one contiguous block of d_Phi).
static spod_status modes_impl(spod_plan_t p, const void* d_X, int nmodes, void* d_Phi, cudaStream_t s,
                              int nrange, const cudaEvent_t* done) {
  {
    Phase ph(p, SPOD_PHASE_MODES, s, 1);
    SPOD_CUDA(launch_mode_coeffs(*p, nmodes, s), "mode coefficient kernel");
    if (p->tensor) {
      SPOD_CUDA(launch_mode_image(*p, nmodes, s), "mode operand image kernel");
      ph.n += 1;
    }
  }
  if (p->qhat_valid) {
    const int nr = std::max(1, std::min(nrange, p->nf));
    for (int r = 0; r < nr; ++r) {
      const int f0 = (int)((int64_t)p->nf * r / nr), f1 = (int)((int64_t)p->nf * (r + 1) / nr);
      Phase ph(p, SPOD_PHASE_MODES, s, 0);
      if (p->tensor) {
        SPOD_CUDA(launch_modes_tc_chunk(*p, 0, p->M, nmodes, d_Phi, s, false, f0, f1), "tensor-core modes kernel");
        ph.n = 1;
      } else {
        SPOD_CUDA(launch_modes_chunk(*p, 0, p->M, nmodes, d_Phi, s, &ph.n, false, f0, f1), "modes kernel");
      }
      if (done) SPOD_CUDA(cudaEventRecord(done[r], s), "range done");
    }
  } else {
    alignas(64) CUtensorMap xmap;
    const CUtensorMap* xm = nullptr;
    if (p->ring_ok) {
      if (spod_status st = make_x_map(p, d_X, &xmap)) return st;
      xm = &xmap;
    }
    for (int64_t m0 = 0; m0 < p->M; m0 += p->chunk_points) {
      const int64_t mc = std::min<int64_t>(p->chunk_points, p->M - m0);
      {
        Phase ph(p, SPOD_PHASE_FFT, s, 1);
        if (spod_status st = run_fft_chunk(p, d_X, xm, m0, mc, s)) return st;
      }
      Phase ph(p, SPOD_PHASE_MODES, s, 0);
      if (p->tensor) {
        SPOD_CUDA(launch_modes_tc_chunk(*p, m0, mc, nmodes, d_Phi, s), "tensor-core modes kernel");
        ph.n = 1;
      } else {
        SPOD_CUDA(launch_modes_chunk(*p, m0, mc, nmodes, d_Phi, s, &ph.n), "modes kernel");
      }
    }
    for (int r = 0; done && r < nrange; ++r) SPOD_CUDA(cudaEventRecord(done[r], s), "range done");
  }
  p->last_stream = s;
  return SPOD_OK;
}

spod_status spod_modes(spod_plan_t p, const void* d_X, int nmodes, void* d_Phi, void* stream) {
  if (spod_status st = check_plan(p)) return st;
  if (!p->fitted) return fail(SPOD_ESTATE, "spod_modes before spod_fit");
  if (nmodes < 1 || nmodes > p->nb) return fail(SPOD_EINVAL, "need 1 <= nmodes <= nb");
  if (spod_status st = check_ptr(d_Phi, "d_Phi")) return st;
  if (!p->qhat_valid) {
    if (spod_status st = check_ptr(d_X, "d_X")) return st;
  }
  DeviceGuard g(p->device);
  return modes_impl(p, d_X, nmodes, d_Phi, static_cast<cudaStream_t>(stream), 1, nullptr);
}

spod_status spod_backward(spod_plan_t p, const double* d_dLdlambda, const void* d_X, void* d_dX, void* stream) {
  if (spod_status st = check_plan(p)) return st;
  if (p->cplx) return fail(SPOD_EUNSUPPORTED, "spod_backward supports real data only");
  if (!p->fitted) return fail(SPOD_ESTATE, "spod_backward before spod_fit");
  if (!d_dLdlambda || reinterpret_cast<uintptr_t>(d_dLdlambda) % 8) return fail(SPOD_EINVAL, "d_dLdlambda NULL or misaligned");
  if (spod_status st = check_ptr(d_dX, "d_dX")) return st;
  if (!p->qhat_valid) {
    if (spod_status st = check_ptr(d_X, "d_X")) return st;
  }
  if (adjoint_smem_bytes(*p) > 227 * 1024) return fail(SPOD_EUNSUPPORTED, "nfft too large for the adjoint kernel");
  DeviceGuard g(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Phase ph(p, SPOD_PHASE_BACKWARD, s, 0);
  SPOD_CUDA(launch_adj_gmat(*p, d_dLdlambda, s), "adjoint G kernel");
  ph.n += 1;
  if (p->tensor) {
    SPOD_CUDA(launch_mode_image(*p, p->adj_cols, s), "adjoint operand image kernel");
    ph.n += 1;
  }
  alignas(64) CUtensorMap xmap;
  const CUtensorMap* xm = nullptr;
  if (!p->qhat_valid && p->ring_ok) {
    if (spod_status st = make_x_map(p, d_X, &xmap)) return st;
    xm = &xmap;
  }
  // per Qhat chunk (recomputed unless the fit left it in place), per column
  // sub-chunk of the plan's R buffer: R = W Qhat G, then the inverse DFT,
  // overlap-add and mean projection of those columns.  R is written and read
  // back one sub-chunk (<= 2 GiB) at a time; no device memory is allocated here.
  const int64_t rw = p->radj_points;
  for (int64_t m0 = 0; m0 < p->M; m0 += p->chunk_points) {
    const int64_t mc = std::min<int64_t>(p->chunk_points, p->M - m0);
    if (!p->qhat_valid) {
      if (spod_status st = run_fft_chunk(p, d_X, xm, m0, mc, s)) return st;
      ph.n += 1;
    }
    for (int64_t s0 = m0; s0 < m0 + mc; s0 += rw) {
      const int64_t sw = std::min<int64_t>(rw, m0 + mc - s0);
      if (p->tensor) {
        SPOD_CUDA(launch_modes_tc_chunk(*p, s0, sw, p->adj_cols, p->d_radj, s, true, 0, -1, s0 - m0, rw, s0),
                  "adjoint R kernel (tensor cores)");
        ph.n += 1;
      } else {
        int nl = 0;
        SPOD_CUDA(launch_modes_chunk(*p, s0, sw, p->adj_cols, p->d_radj, s, &nl, true, 0, -1, s0 - m0, rw, s0),
                  "adjoint R kernel");
        ph.n += nl;
      }
      SPOD_CUDA(launch_adjoint_chunk(*p, p->d_radj, rw, s0, s0, sw, d_dX, s), "adjoint kernel");
      ph.n += 1;
    }
  }
  p->last_stream = s;
  return SPOD_OK;
}

// Datasets from and to host memory, one after another through the plan.
// The host link (~200 GB/s each way, ~340 GB/s both ways at once) is the
// bound, so the copies run on two plan-owned streams beside the compute
// stream: dataset i + 1's X goes up while dataset i's modes come down, from
// two staging pairs used in turn; each dataset's modes are computed in
// kRanges frequency ranges, and a range goes down while the next one is
// computed.
constexpr int kRanges = 8;

static spod_status grow(void** buf, size_t* have, size_t need, const char* what) {
  if (*have >= need) return SPOD_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *have = 0;
  if (cudaMalloc(buf, need) != cudaSuccess) {
    cudaGetLastError();
    return fail(SPOD_ENOMEM, what);
  }
  *have = need;
  return SPOD_OK;
}

static spod_status run_host_impl(spod_plan_t p, int n, const void* const* h_X, int nmodes, void* const* h_Phi,
                                 double* const* h_lambda, cudaStream_t s) {
  const size_t el = elem_bytes(p->desc.in_dtype);
  const size_t xb = (size_t)p->nt * p->M * el;
  const size_t eb = p->f64 ? 16 : 8;            // one complex element of Phi
  const size_t fb = (size_t)nmodes * p->M * eb; // Phi bytes of one frequency
  const size_t pb = (size_t)p->nf * fb;
  const int nbuf = n > 1 ? 2 : 1;
  SPOD_CUDA(cudaStreamSynchronize(s), "stream synchronize");   // staging may be reallocated
  // staging pair 0 (kept across calls), pair 1 only for several datasets
  if (spod_status st = grow(&p->d_xstage, &p->xstage_bytes, xb, "X staging")) return st;
  if (nmodes > 0) {
    if (spod_status st = grow(&p->d_phistage, &p->phistage_bytes, pb, "Phi staging")) return st;
  }
  const size_t lb = sizeof(double) * (size_t)p->nf * p->nb;
  if (h_lambda) {
    if (spod_status st = grow(&p->d_lamstage, &p->lamstage_bytes, lb * n, "eigenvalue staging")) return st;
  }
  if (nbuf == 2) {
    if (spod_status st = grow(&p->d_xstage2, &p->xstage2_bytes, xb, "X staging")) return st;
    if (nmodes > 0) {
      if (spod_status st = grow(&p->d_phistage2, &p->phistage2_bytes, pb, "Phi staging")) return st;
    }
  }
  if (!p->h2d_stream) SPOD_CUDA(cudaStreamCreateWithFlags(&p->h2d_stream, cudaStreamNonBlocking), "copy stream");
  if (!p->d2h_stream) SPOD_CUDA(cudaStreamCreateWithFlags(&p->d2h_stream, cudaStreamNonBlocking), "copy stream");
  // events: x_ready[2], x_free[2], phi_free[2], start, range_done[2][kRanges]
  const size_t nev = 7 + 2 * kRanges;
  while (p->host_ev.size() < nev) {
    cudaEvent_t e;
    SPOD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    p->host_ev.push_back(e);
  }
  cudaEvent_t* x_ready = &p->host_ev[0];
  cudaEvent_t* x_free = &p->host_ev[2];
  cudaEvent_t* phi_free = &p->host_ev[4];
  cudaEvent_t start = p->host_ev[6];
  cudaEvent_t* range_done = &p->host_ev[7];
  void* xs[2] = {p->d_xstage, p->d_xstage2};
  void* ps[2] = {p->d_phistage, p->d_phistage2};
  cudaStream_t up = p->h2d_stream, down = p->d2h_stream;
  SPOD_CUDA(cudaEventRecord(start, s), "event");
  SPOD_CUDA(cudaStreamWaitEvent(up, start, 0), "wait");
  SPOD_CUDA(cudaStreamWaitEvent(down, start, 0), "wait");
  for (int i = 0; i < n; ++i) {
    const int b = i % nbuf;
    // X of dataset i into staging b once dataset i - 2 no longer reads it
    if (i >= nbuf) SPOD_CUDA(cudaStreamWaitEvent(up, x_free[b], 0), "wait");
    SPOD_CUDA(cudaMemcpyAsync(xs[b], h_X[i], xb, cudaMemcpyHostToDevice, up), "copy X to device");
    SPOD_CUDA(cudaEventRecord(x_ready[b], up), "event");
    SPOD_CUDA(cudaStreamWaitEvent(s, x_ready[b], 0), "wait");
    if (spod_status st = fit_impl(p, xs[b], s, p->chunk_points)) return st;
    // eigenvalues to device staging (a pageable host copy here would stall the pipeline)
    if (h_lambda && h_lambda[i])
      SPOD_CUDA(cudaMemcpyAsync(static_cast<char*>(p->d_lamstage) + lb * i, p->d_lam, lb, cudaMemcpyDeviceToDevice, s),
                "stage lambda");
    if (nmodes > 0) {
      // Phi staging b once dataset i - 2's modes have gone down
      if (i >= nbuf) SPOD_CUDA(cudaStreamWaitEvent(s, phi_free[b], 0), "wait");
      if (spod_status st = modes_impl(p, xs[b], nmodes, ps[b], s, kRanges, range_done + b * kRanges)) return st;
      for (int r = 0; r < kRanges; ++r) {
        const int nr = std::min(kRanges, p->nf);
        if (r >= nr) break;
        const int64_t f0 = (int64_t)p->nf * r / nr, f1 = (int64_t)p->nf * (r + 1) / nr;
        SPOD_CUDA(cudaStreamWaitEvent(down, range_done[b * kRanges + r], 0), "wait");
        SPOD_CUDA(cudaMemcpyAsync(static_cast<char*>(h_Phi[i]) + f0 * fb, static_cast<const char*>(ps[b]) + f0 * fb,
                                  (f1 - f0) * fb, cudaMemcpyDeviceToHost, down), "copy Phi to host");
      }
      SPOD_CUDA(cudaEventRecord(phi_free[b], down), "event");
    }
    SPOD_CUDA(cudaEventRecord(x_free[b], s), "event");
  }
  SPOD_CUDA(cudaEventRecord(start, up), "event");
  SPOD_CUDA(cudaStreamWaitEvent(s, start, 0), "join");
  SPOD_CUDA(cudaEventRecord(start, down), "event");
  SPOD_CUDA(cudaStreamWaitEvent(s, start, 0), "join");
  for (int i = 0; h_lambda && i < n; ++i)
    if (h_lambda[i])
      SPOD_CUDA(cudaMemcpyAsync(h_lambda[i], static_cast<const char*>(p->d_lamstage) + lb * i, lb,
                                cudaMemcpyDeviceToHost, s), "copy lambda to host");
  SPOD_CUDA(cudaStreamSynchronize(s), "stream synchronize");
  return read_flags(p);
}

spod_status spod_run_host(spod_plan_t p, const void* h_X, int nmodes, void* h_Phi, double* h_lambda,
                          void* stream) {
  if (spod_status st = check_plan(p)) return st;
  if (!h_X) return fail(SPOD_EINVAL, "h_X is NULL");
  if (nmodes < 0 || nmodes > p->nb) return fail(SPOD_EINVAL, "need 0 <= nmodes <= nb");
  if (nmodes > 0 && !h_Phi) return fail(SPOD_EINVAL, "h_Phi is NULL");
  DeviceGuard g(p->device);
  return run_host_impl(p, 1, &h_X, nmodes, &h_Phi, &h_lambda, static_cast<cudaStream_t>(stream));
}

spod_status spod_run_host_many(spod_plan_t p, int n, const void* const* h_X, int nmodes, void* const* h_Phi,
                               double* const* h_lambda, void* stream) {
  if (spod_status st = check_plan(p)) return st;
  if (n < 1 || !h_X) return fail(SPOD_EINVAL, "need n >= 1 and h_X");
  if (nmodes < 0 || nmodes > p->nb) return fail(SPOD_EINVAL, "need 0 <= nmodes <= nb");
  for (int i = 0; i < n; ++i) {
    if (!h_X[i]) return fail(SPOD_EINVAL, "h_X[i] is NULL");
    if (nmodes > 0 && (!h_Phi || !h_Phi[i])) return fail(SPOD_EINVAL, "h_Phi[i] is NULL");
  }
  DeviceGuard g(p->device);
  return run_host_impl(p, n, h_X, nmodes, h_Phi, h_lambda, static_cast<cudaStream_t>(stream));
}

// Out-of-core pipeline: X and Phi stay in pinned host memory; column tiles of
// w points are gathered over the host link by a copy kernel (on the plan's
// upload stream) into two device tile buffers used in turn, and the fit runs
// tile by tile (mean, FFT, Gram of tile c while tile c + 1 arrives); after
// the eigen-solve the tiles are gathered again, their Qhat recomputed and
// their modes written into two device Phi tiles, each scattered back to the
// host while the next one is computed.  Device memory: the plan's workspace
// and the four tile buffers.
spod_status spod_run_host_ooc(spod_plan_t p, const void* h_X, int nmodes, void* h_Phi, double* h_lambda,
                              int64_t tile_points, void* stream) {
  if (spod_status st = check_plan(p)) return st;
  if (!h_X) return fail(SPOD_EINVAL, "h_X is NULL");
  if (nmodes < 0 || nmodes > p->nb) return fail(SPOD_EINVAL, "need 0 <= nmodes <= nb");
  if (nmodes > 0 && !h_Phi) return fail(SPOD_EINVAL, "h_Phi is NULL");
  if (tile_points < 0) return fail(SPOD_EINVAL, "tile_points must be >= 0");
  DeviceGuard g(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the kernels read and write the host arrays directly: pinned memory through
  // its device alias, pageable memory only where the device reads it through
  // the host's page tables
  int pageable = 0;
  if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, p->device) != cudaSuccess) {
    cudaGetLastError();
    pageable = 0;
  }
  auto device_alias = [&](void* h, void** d) {
    if (cudaHostGetDevicePointer(d, h, 0) == cudaSuccess) return true;
    cudaGetLastError();
    *d = h;
    return pageable != 0;
  };
  void *dXh = nullptr, *dPh = nullptr;
  if (!device_alias(const_cast<void*>(h_X), &dXh))
    return fail(SPOD_EINVAL, "h_X must be pinned host memory (cudaHostAlloc / cudaHostRegister)");
  if (nmodes > 0 && !device_alias(h_Phi, &dPh))
    return fail(SPOD_EINVAL, "h_Phi must be pinned host memory (cudaHostAlloc / cudaHostRegister)");
  const int64_t M = p->M, nt = p->nt;
  int64_t w = tile_points ? tile_points : ((M + 3) / 4 + 63) / 64 * 64;
  // whole multiples of 64 points (16-byte aligned tile rows), within the plan's Qhat chunk
  w = std::min<int64_t>(std::max<int64_t>(64, (w + 63) / 64 * 64), p->chunk_points);
  const int64_t ntile = (M + w - 1) / w;
  const size_t el = elem_bytes(p->desc.in_dtype);
  const size_t eb = p->f64 ? 16 : 8;
  const size_t xtb = (size_t)nt * w * el, ptb = (size_t)p->nf * nmodes * w * eb;
  if (!p->h2d_stream) SPOD_CUDA(cudaStreamCreateWithFlags(&p->h2d_stream, cudaStreamNonBlocking), "copy stream");
  if (!p->d2h_stream) SPOD_CUDA(cudaStreamCreateWithFlags(&p->d2h_stream, cudaStreamNonBlocking), "copy stream");
  while (p->host_ev.size() < 16) {
    cudaEvent_t e;
    SPOD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    p->host_ev.push_back(e);
  }
  cudaEvent_t* ready = &p->host_ev[0];      // [2] X tile arrived
  cudaEvent_t* xfree = &p->host_ev[2];      // [2] X tile consumed
  cudaEvent_t* pready = &p->host_ev[4];     // [2] Phi tile written
  cudaEvent_t* pfree = &p->host_ev[6];      // [2] Phi tile sent
  cudaEvent_t start = p->host_ev[8];
  cudaStream_t up = p->h2d_stream, down = p->d2h_stream;
  void *xt[2] = {nullptr, nullptr}, *pt[2] = {nullptr, nullptr};
  auto release = [&]() {
    for (int b = 0; b < 2; ++b) {
      if (xt[b]) cudaFreeAsync(xt[b], s);
      if (pt[b]) cudaFreeAsync(pt[b], s);
    }
    p->x_ld = p->x_off = p->phi_ld = p->phi_off = 0;
  };
  for (int b = 0; b < 2; ++b) {
    if (cudaMallocAsync(&xt[b], xtb, s) != cudaSuccess || (nmodes > 0 && cudaMallocAsync(&pt[b], ptb, s) != cudaSuccess)) {
      cudaGetLastError();
      release();
      return fail(SPOD_ENOMEM, "out-of-core tile buffers");
    }
  }
  spod_status st = SPOD_OK;
  auto ck = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && st == SPOD_OK) st = cuda_fail(e, what);
    return st == SPOD_OK;
  };
  ck(cudaEventRecord(start, s), "event");
  ck(cudaStreamWaitEvent(up, start, 0), "wait");
  ck(cudaStreamWaitEvent(down, start, 0), "wait");
  auto gather = [&](int64_t c, int b, int use) {
    const int64_t c0 = c * w, wc = std::min<int64_t>(w, M - c0);
    if (use >= 2) ck(cudaStreamWaitEvent(up, xfree[b], 0), "wait");
    // the columns past the last point read as zeros, as TMA's out-of-range fill does for untiled data
    ck(launch_copy2d(xt[b], w * el, static_cast<const char*>(dXh) + c0 * el, M * el, wc * el, w * el, nt,
                     p->num_sms, up),
       "gather X tile");
    ck(cudaEventRecord(ready[b], up), "event");
    ck(cudaStreamWaitEvent(s, ready[b], 0), "wait");
  };
  // ---- fit
  p->fitted = false;
  p->qhat_valid = false;
  p->x_ld = w;
  ck(cudaMemsetAsync(p->d_flags, 0, sizeof(unsigned), s), "clear flags");      // [1] is the wait bound
  if (!p->desc.subtract_mean) ck(cudaMemsetAsync(p->d_mu, 0, sizeof(double) * M * (p->cplx ? 2 : 1), s), "zero mean");
  int use = 0;
  for (int64_t c = 0; c < ntile && st == SPOD_OK; ++c, ++use) {
    const int b = use & 1;
    const int64_t c0 = c * w, wc = std::min<int64_t>(w, M - c0);
    gather(c, b, use);
    p->x_off = c0;
    if (p->desc.subtract_mean && !p->mean_fold) ck(launch_mean(*p, xt[b], c0, wc, s), "mean kernel");
    alignas(64) CUtensorMap xmap;
    const CUtensorMap* xm = nullptr;
    if (p->ring_ok && st == SPOD_OK) {
      if ((st = make_x_map(p, xt[b], &xmap)) != SPOD_OK) break;
      xm = &xmap;
    }
    if (st == SPOD_OK) st = run_fft_chunk(p, xt[b], xm, c0, wc, s);
    if (p->tensor) ck(launch_gram_tc_chunk(*p, wc, c == 0, s), "tensor-core gram kernel");
    else ck(launch_gram_chunk(*p, wc, c == 0, s), "gram kernel");
    ck(cudaEventRecord(xfree[b], s), "event");
  }
  if (p->tensor) ck(launch_gram_tc_finish(*p, s), "gram finish kernel");
  else ck(launch_gram_reduce(*p, s), "gram reduce kernel");
  ck(launch_eig_tridiag(*p, s), "eigen-solver kernel");
  if (st == SPOD_OK) {
    p->fitted = true;
    p->partial = false;
  }
  if (h_lambda)
    ck(cudaMemcpyAsync(h_lambda, p->d_lam, sizeof(double) * (size_t)p->nf * p->nb, cudaMemcpyDeviceToHost, s),
       "copy lambda to host");
  // ---- modes
  if (nmodes > 0 && st == SPOD_OK) {
    ck(launch_mode_coeffs(*p, nmodes, s), "mode coefficient kernel");
    if (p->tensor) ck(launch_mode_image(*p, nmodes, s), "mode operand image kernel");
    p->phi_ld = w;
    for (int64_t c = 0; c < ntile && st == SPOD_OK; ++c, ++use) {
      const int b = use & 1, pb = (int)(c & 1);
      const int64_t c0 = c * w, wc = std::min<int64_t>(w, M - c0);
      gather(c, b, use);
      p->x_off = c0;
      alignas(64) CUtensorMap xmap;
      const CUtensorMap* xm = nullptr;
      if (p->ring_ok) {
        if ((st = make_x_map(p, xt[b], &xmap)) != SPOD_OK) break;
        xm = &xmap;
      }
      if ((st = run_fft_chunk(p, xt[b], xm, c0, wc, s)) != SPOD_OK) break;
      ck(cudaEventRecord(xfree[b], s), "event");
      if (c >= 2) ck(cudaStreamWaitEvent(s, pfree[pb], 0), "wait");
      p->phi_off = c0;
      int nl = 0;
      if (p->tensor) ck(launch_modes_tc_chunk(*p, c0, wc, nmodes, pt[pb], s), "tensor-core modes kernel");
      else ck(launch_modes_chunk(*p, c0, wc, nmodes, pt[pb], s, &nl), "modes kernel");
      ck(cudaEventRecord(pready[pb], s), "event");
      ck(cudaStreamWaitEvent(down, pready[pb], 0), "wait");
      ck(launch_copy2d(static_cast<char*>(dPh) + c0 * eb, M * eb, pt[pb], w * eb, wc * eb, wc * eb,
                       (int64_t)p->nf * nmodes, p->num_sms, down),
         "scatter Phi tile");
      ck(cudaEventRecord(pfree[pb], down), "event");
    }
  }
  ck(cudaEventRecord(start, up), "event");
  ck(cudaStreamWaitEvent(s, start, 0), "join");
  ck(cudaEventRecord(start, down), "event");
  ck(cudaStreamWaitEvent(s, start, 0), "join");
  release();
  p->qhat_valid = false;
  p->last_stream = s;
  if (st != SPOD_OK) return st;
  SPOD_CUDA(cudaStreamSynchronize(s), "stream synchronize");
  return read_flags(p);
}

// Validation shared by the expansion-coefficient entries.
static spod_status check_coeff_args(spod_plan_t p, const void* d_Phi, int nmodes, int nmodes_r, int nfreq_r,
                                    const int* h_freqs) {
  if (!p->fitted) return fail(SPOD_ESTATE, "expansion coefficients before spod_fit");
  if (p->cplx) return fail(SPOD_EUNSUPPORTED, "expansion coefficients support real data only");
  if (p->f64 ? p->desc.in_dtype != SPOD_F64 : p->desc.in_dtype != SPOD_F32)
    return fail(SPOD_EUNSUPPORTED, "expansion coefficients need F64 data with FP64 precision or F32 data otherwise");
  if (spod_status st = check_ptr(d_Phi, "d_Phi")) return st;
  if (nmodes < 1 || nmodes > p->nb || nmodes_r < 1 || nmodes_r > nmodes)
    return fail(SPOD_EINVAL, "need 1 <= nmodes_r <= nmodes <= nb");
  if (nfreq_r < 1 || nfreq_r > p->nf || !h_freqs) return fail(SPOD_EINVAL, "need 1 <= nfreq_r <= nf and h_freqs");
  std::vector<char> seen(p->nf, 0);
  for (int j = 0; j < nfreq_r; ++j) {
    if (h_freqs[j] < 0 || h_freqs[j] >= p->nf) return fail(SPOD_EINVAL, "h_freqs entry outside 0 .. nf-1");
    if (seen[h_freqs[j]]++) return fail(SPOD_EINVAL, "h_freqs entries must be distinct");
  }
  if (coeff_basis_size(*p, nmodes_r, nfreq_r, h_freqs) > 4096)
    return fail(SPOD_EUNSUPPORTED, "more than 4096 real basis vectors");
  return SPOD_OK;
}

spod_status spod_coeffs(spod_plan_t p, const void* d_X, const void* d_Phi, int nmodes, int nmodes_r, int nfreq_r,
                        const int* h_freqs, double* d_A, void* stream) {
  if (spod_status st = check_plan(p)) return st;
  if (spod_status st = check_coeff_args(p, d_Phi, nmodes, nmodes_r, nfreq_r, h_freqs)) return st;
  if (spod_status st = check_ptr(d_X, "d_X")) return st;
  if (spod_status st = check_ptr(d_A, "d_A")) return st;
  DeviceGuard g(p->device);
  SPOD_CUDA(launch_coeffs(*p, d_X, d_Phi, nmodes, nmodes_r, nfreq_r, h_freqs, d_A, static_cast<cudaStream_t>(stream)),
            "expansion coefficients");
  return SPOD_OK;
}

spod_status spod_reconstruct(spod_plan_t p, const void* d_Phi, int nmodes, int nmodes_r, int nfreq_r,
                             const int* h_freqs, const double* d_A, void* d_Xrec, void* stream) {
  if (spod_status st = check_plan(p)) return st;
  if (spod_status st = check_coeff_args(p, d_Phi, nmodes, nmodes_r, nfreq_r, h_freqs)) return st;
  if (spod_status st = check_ptr(d_A, "d_A")) return st;
  if (spod_status st = check_ptr(d_Xrec, "d_Xrec")) return st;
  DeviceGuard g(p->device);
  SPOD_CUDA(launch_reconstruct(*p, d_Phi, nmodes, nmodes_r, nfreq_r, h_freqs, d_A, d_Xrec,
                               static_cast<cudaStream_t>(stream)),
            "reconstruction");
  return SPOD_OK;
}

spod_status spod_plan_get_tuning(spod_plan_t p, spod_tuning* t) {
  if (spod_status st = check_plan(p)) return st;
  if (!t) return fail(SPOD_EINVAL, "tuning is NULL");
  t->gram_splits = p->gram_splits;
  t->gram_splits_max = p->gram_splits_max;
  t->gram_flush_blocks = p->gram_flush;
  t->modes_ctas = p->modes_ctas;
  t->eig_max_iter = p->eig_max_iter;
  t->wait_timeout_us = p->wait_timeout_us;
  t->wait_selftest = p->wait_selftest;
  t->fft_tile_points = p->pipe_ok ? p->pipe_tp : 0;
  return SPOD_OK;
}

spod_status spod_plan_set_tuning(spod_plan_t p, const spod_tuning* t) {
  if (spod_status st = check_plan(p)) return st;
  if (!t) return fail(SPOD_EINVAL, "tuning is NULL");
  if (t->gram_splits < 0 || t->gram_splits > p->gram_splits_max)
    return fail(SPOD_EINVAL, "gram_splits must be in 1..gram_splits_max");
  if (t->gram_flush_blocks < 0 || t->gram_flush_blocks > 64) return fail(SPOD_EINVAL, "gram_flush_blocks must be in 1..64");
  if (t->modes_ctas < 0 || t->modes_ctas > 4096) return fail(SPOD_EINVAL, "modes_ctas must be in 0..4096");
  if (t->eig_max_iter < 0 || t->eig_max_iter > 1000) return fail(SPOD_EINVAL, "eig_max_iter must be in 0..1000");
  if (t->wait_timeout_us < 0 || t->wait_timeout_us > 4000000)
    return fail(SPOD_EINVAL, "wait_timeout_us must be in 0..4000000");
  if (t->wait_selftest < 0 || t->wait_selftest > 1) return fail(SPOD_EINVAL, "wait_selftest must be 0 or 1");
  if (t->fft_tile_points != 0 && (p->pipe_ok ? t->fft_tile_points != p->pipe_tp : true)) {
    if (!p->pipe_ok) return fail(SPOD_EINVAL, "fft_tile_points: this plan does not use the pipelined FFT");
    if (t->fft_tile_points != 16 && t->fft_tile_points != 32)
      return fail(SPOD_EINVAL, "fft_tile_points must be 16 or 32");
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    const size_t sm = fft_pipe_smem_bytes(*p, t->fft_tile_points);
    if (sm == 0 || sm > (size_t)optin)
      return fail(SPOD_EINVAL, "fft_tile_points: no form of the pipelined FFT with that tile for this plan");
  }
  if (t->wait_timeout_us != p->wait_timeout_us) {
    DeviceGuard g(p->device);
    const unsigned us = (unsigned)t->wait_timeout_us;
    SPOD_CUDA(cudaMemcpy(p->d_flags + 1, &us, sizeof(us), cudaMemcpyHostToDevice), "set the wait bound");
    p->wait_timeout_us = t->wait_timeout_us;
  }
  if (t->gram_splits) p->gram_splits = t->gram_splits;
  if (t->gram_flush_blocks) p->gram_flush = t->gram_flush_blocks;
  p->modes_ctas = t->modes_ctas;
  p->eig_max_iter = t->eig_max_iter;
  p->wait_selftest = t->wait_selftest;
  if (t->fft_tile_points) p->pipe_tp = t->fft_tile_points;
  ++p->version;
  return SPOD_OK;
}

spod_status spod_profile_enable(spod_plan_t p, int enable) {
  if (spod_status st = check_plan(p)) return st;
  p->prof = enable != 0;
  return SPOD_OK;
}

spod_status spod_profile_read(spod_plan_t p, double* ms, int64_t* launches) {
  if (spod_status st = check_plan(p)) return st;
  DeviceGuard g(p->device);
  double acc[SPOD_NPHASES] = {0};
  spod_status st = SPOD_OK;
  for (auto& r : p->recs) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess && st == SPOD_OK) st = cuda_fail(e, "phase timing");
    acc[r.phase] += t;
    p->ev_free.push_back(r.a);
    p->ev_free.push_back(r.b);
  }
  p->recs.clear();
  for (int i = 0; i < SPOD_NPHASES; ++i) {
    if (ms) ms[i] = acc[i];
    if (launches) launches[i] = p->launches[i];
    p->launches[i] = 0;
  }
  return st;
}

// ---- spod_fit_batch: the n fits captured once into a CUDA graph with one
// branch per dataset (independent plans run concurrently and fill the GPU
// when a dataset alone would not), then relaunched while the plans, their
// launch parameters and the inputs stay the same.
namespace {
struct BatchGraph {
  int device = -1;
  std::vector<uint64_t> key;                 // (uid, version, X) per plan
  cudaGraphExec_t exec = nullptr;
  cudaStream_t origin = nullptr;             // capture stream
  std::vector<cudaStream_t> side;            // one branch per dataset
  std::vector<cudaEvent_t> ev;               // fork + joins
};
std::mutex g_batch_mu;
std::vector<BatchGraph> g_batch;             // one cached graph per device

spod_status batch_resources(BatchGraph& bg, int n) {
  if (!bg.origin) SPOD_CUDA(cudaStreamCreateWithFlags(&bg.origin, cudaStreamNonBlocking), "batch stream");
  while ((int)bg.side.size() < n) {
    cudaStream_t st;
    SPOD_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "batch stream");
    bg.side.push_back(st);
  }
  while ((int)bg.ev.size() < n + 1) {
    cudaEvent_t e;
    SPOD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "batch event");
    bg.ev.push_back(e);
  }
  return SPOD_OK;
}
}  // namespace

spod_status spod_fit_batch(spod_plan_t* plans, const void* const* d_X, int n, void* stream) {
  if (!plans || !d_X || n < 0) return fail(SPOD_EINVAL, "bad batch arguments");
  if (n == 0) return SPOD_OK;
  std::vector<uint64_t> key;
  for (int i = 0; i < n; ++i) {
    if (spod_status st = check_plan(plans[i])) return st;
    if (spod_status st = check_ptr(d_X[i], "d_X[i]")) return st;
    if (plans[i]->device != plans[0]->device) return fail(SPOD_EINVAL, "batch plans must share one device");
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return fail(SPOD_EINVAL, "a plan appears twice in the batch");
    key.push_back(plans[i]->uid);
    key.push_back(plans[i]->version);
    key.push_back((uint64_t)reinterpret_cast<uintptr_t>(d_X[i]));
  }
  DeviceGuard g(plans[0]->device);
  if (!g.ok) return fail(SPOD_ECUDA, "cannot select the plans' device");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_batch_mu);
  BatchGraph* bgp = nullptr;
  for (auto& b : g_batch)
    if (b.device == plans[0]->device) bgp = &b;
  if (!bgp) {
    g_batch.emplace_back();
    bgp = &g_batch.back();
    bgp->device = plans[0]->device;
  }
  BatchGraph& bg = *bgp;
  if (!(bg.exec && bg.key == key)) {
    if (spod_status st = batch_resources(bg, n)) return st;
    if (bg.exec) { cudaGraphExecDestroy(bg.exec); bg.exec = nullptr; }
    bg.key.clear();
    // the work must be in stream order after anything already queued on `stream`
    // only at launch; capture happens on a private stream
    SPOD_CUDA(cudaStreamBeginCapture(bg.origin, cudaStreamCaptureModeThreadLocal), "begin graph capture");
    spod_status st = SPOD_OK;
    std::string msg;
    std::vector<int> prof(n);
    if (cudaEventRecord(bg.ev[0], bg.origin) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "fork event");
    for (int i = 0; i < n && st == SPOD_OK; ++i) {
      prof[i] = plans[i]->prof;
      plans[i]->prof = 0;                    // phase events stay outside the graph
      if (cudaStreamWaitEvent(bg.side[i], bg.ev[0], 0) != cudaSuccess) {
        st = cuda_fail(cudaGetLastError(), "fork");
      } else {
        st = spod_fit(plans[i], d_X[i], bg.side[i]);
        if (st == SPOD_OK && (cudaEventRecord(bg.ev[i + 1], bg.side[i]) != cudaSuccess ||
                              cudaStreamWaitEvent(bg.origin, bg.ev[i + 1], 0) != cudaSuccess))
          st = cuda_fail(cudaGetLastError(), "join");
      }
      plans[i]->prof = prof[i];
    }
    if (st != SPOD_OK) msg = spod_last_error();
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(bg.origin, &graph);
    if (st != SPOD_OK) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return fail(st, "batch capture: " + msg);
    }
    if (ec != cudaSuccess) return cuda_fail(ec, "end graph capture");
    const cudaError_t ei = cudaGraphInstantiate(&bg.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) { bg.exec = nullptr; return cuda_fail(ei, "instantiate graph"); }
    bg.key = key;
  }
  SPOD_CUDA(cudaGraphLaunch(bg.exec, s), "graph launch");
  for (int i = 0; i < n; ++i) plans[i]->last_stream = s;
  return SPOD_OK;
}

// ---- spod_plan_autotune: time spod_fit under candidate launch shapes on
// the caller's input and keep the fastest: the pipelined FFT's tile width,
// then the Gram's CTA count.  Only how work is split across CTAs is
// searched; the FP32 accumulation interval (gram_flush_blocks), which
// changes rounding, is left as it is.
spod_status spod_plan_autotune(spod_plan_t p, const void* d_X, void* stream, spod_tuning* chosen) {
  if (spod_status st = check_plan(p)) return st;
  if (spod_status st = check_ptr(d_X, "d_X")) return st;
  DeviceGuard g(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int sms = p->num_sms > 0 ? p->num_sms : 148;
  std::vector<int> cand;
  if (p->tensor) {
    for (int c : {sms, sms / 2, sms + sms / 2, 2 * sms})
      if (c >= 1 && c <= p->gram_splits_max) cand.push_back(c);
  } else {
    const int d = p->gram_splits;
    for (int c : {d, d / 2, d * 2, d * 4, (d * 3) / 2})
      if (c >= 1 && c <= p->gram_splits_max) cand.push_back(c);
  }
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  // FFT tile widths with a compiled form that fits (pipelined FFT only)
  std::vector<int> tiles;
  if (p->pipe_ok) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    for (int tp : {16, 32}) {
      const size_t sm = fft_pipe_smem_bytes(*p, tp);
      if (sm > 0 && sm <= (size_t)optin) tiles.push_back(tp);
    }
  }
  const int keep_splits = p->gram_splits, keep_tp = p->pipe_tp;
  const int prof = p->prof;
  p->prof = 0;
  cudaEvent_t e0, e1;
  SPOD_CUDA(cudaEventCreate(&e0), "event");
  SPOD_CUDA(cudaEventCreate(&e1), "event");
  spod_status st = SPOD_OK;
  // one warm-up fit, then two timed ones
  auto time_fit = [&](float& ms) -> spod_status {
    if (spod_status r = spod_fit(p, d_X, stream)) return r;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 2; ++r)
      if (spod_status q = spod_fit(p, d_X, stream)) return q;
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return cuda_fail(cudaGetLastError(), "autotune timing");
    cudaEventElapsedTime(&ms, e0, e1);
    return SPOD_OK;
  };
  // the FFT tile first (at the current Gram split), then the Gram split
  float best = 1e30f;
  int best_tp = keep_tp;
  for (int tp : tiles) {
    if (st != SPOD_OK) break;
    p->pipe_tp = tp;
    ++p->version;
    float ms = 0.f;
    st = time_fit(ms);
    if (st == SPOD_OK && ms < best) { best = ms; best_tp = tp; }
  }
  p->pipe_tp = st == SPOD_OK ? best_tp : keep_tp;
  best = 1e30f;
  int best_c = keep_splits;
  for (int c : cand) {
    if (st != SPOD_OK) break;
    p->gram_splits = c;
    float ms = 0.f;
    st = time_fit(ms);
    if (st == SPOD_OK && ms < best) { best = ms; best_c = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->gram_splits = st == SPOD_OK ? best_c : keep_splits;
  if (st != SPOD_OK) p->pipe_tp = keep_tp;
  p->prof = prof;
  ++p->version;
  if (st != SPOD_OK) return st;
  if (chosen) spod_plan_get_tuning(p, chosen);
  return SPOD_OK;
}

}  // extern "C"
