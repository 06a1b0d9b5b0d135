// C ABI of the GB300 NB-LDPC decoders, FFT-SPA side (Alg. 1; declarations and
// contracts in include/nbldpc.h): the launch shape of a code (check-node form,
// degree buckets, block size, shared memory, message slot), stream-ordered
// launches of the FFT-SPA kernels, device- and host-buffer entry points.
#include "nbldpc.h"

#include "fftspa_kernels.cuh"
#include "host_internal.h"

static_assert(sizeof(nbldpc::FftParams) < 4000, "kernel parameter space");

using namespace nbldpc_host;

namespace nbldpc {   // defined in fftspa.cu, one translation unit per field order
const void* fft_kernel_q2(int dc, int dv, int* threads);
const void* fft_kernel_q4(int dc, int dv, int* threads);
const void* fft_kernel_q8(int dc, int dv, int* threads);
const void* fft_kernel_q16(int dc, int dv, int* threads);
const void* fft_kernel_q32(int dc, int dv, int* threads);
const void* fft_kernel_q64(int dc, int dv, int* threads);
const void* fft_kernel_q128(int dc, int dv, int* threads);
const void* fft_kernel_q256(int dc, int dv, int* threads);
}  // namespace nbldpc

namespace {

const void* fft_kernel_for(int q, int dc, int dv, int* threads = nullptr) {
  switch (q) {
    case 2: return nbldpc::fft_kernel_q2(dc, dv, threads);
    case 4: return nbldpc::fft_kernel_q4(dc, dv, threads);
    case 8: return nbldpc::fft_kernel_q8(dc, dv, threads);
    case 16: return nbldpc::fft_kernel_q16(dc, dv, threads);
    case 32: return nbldpc::fft_kernel_q32(dc, dv, threads);
    case 64: return nbldpc::fft_kernel_q64(dc, dv, threads);
    case 128: return nbldpc::fft_kernel_q128(dc, dv, threads);
    case 256: return nbldpc::fft_kernel_q256(dc, dv, threads);
  }
  return nullptr;
}

// Largest field order whose codes take the lane-per-edge check-node form at
// every check degree (compile-time tuning knob).  Measured on GB300 (Mbit/s,
// lane per edge against distributed with 4 elements per lane): GF(4) (2,4)
// N=48 1336 vs 1117, GF(8) (2,4) N=512 1441 vs 1467, GF(16) (2,4) N=1024
// 1432 vs 1759, GF(32) (3,6) N=600 408 vs 588.
#ifndef NBLDPC_FFT_LANE_MAXQ
#define NBLDPC_FFT_LANE_MAXQ 4
#endif

bool g_fft_attr_done[64][8][3][3] = {};   // device, log2(q) - 1, check-node form, column-degree bucket

}  // namespace

// Launch shape of the FFT-SPA kernel for a code: check-node form and degree
// buckets, block size (one frame per SM), shared memory (code blob, decisions,
// control word, and for the lane-per-edge form one transformed vector per
// lane), resident blocks, message slot of nnz * q floats.
int nbldpc_host::fft_configure(nbldpc_code* c) {
  // check-node form: lane per edge (dc 0: check degree <= 32) for small fields
  // and for q <= 64 codes with a check of degree > 8; otherwise the
  // distributed form with the check degree bucket 4 or 8
  const bool lane_form = c->q <= NBLDPC_FFT_LANE_MAXQ || (c->q <= 64 && c->dmax > 8);
  const int dc = lane_form ? (c->dmax <= 32 ? 0 : -1) : (c->dmax <= 4 ? 4 : (c->dmax <= 8 ? 8 : -1));
  const int dv = c->vmax <= 2 ? 2 : (c->vmax <= 4 ? 4 : (c->vmax <= 8 ? 8 : 0));
  if (dc < 0 || !dv) return NBLDPC_ERR_UNSUPPORTED;
  int threads = 0;
  const void* k = fft_kernel_for(c->q, dc, dv, &threads);
  if (!k) return NBLDPC_ERR_UNSUPPORTED;
  int dev = 0, sms = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return NBLDPC_ERR_CUDA;
  if (dev < 0 || dev >= 64) return NBLDPC_ERR_CUDA;
  Plan pl{};
  pl.fpb = 1;
  pl.threads = threads;
  pl.blob_cap = (int)round_up((size_t)c->off.fft_bytes, 16);
  pl.n_cap = (int)round_up((size_t)c->n, 16);
  const int w_area = dc == 0 ? threads * c->q * (int)sizeof(float) : 0;   // one transformed vector per lane
  pl.slot_smem = pl.smem = (int)round_up((size_t)(pl.blob_cap + pl.n_cap + 16), 256) + w_area;
  if (pl.smem > optin) return NBLDPC_ERR_UNSUPPORTED;
  {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    bool& done = g_fft_attr_done[dev][nbldpc::ilog2(c->q) - 1][dc == 0 ? 0 : (dc == 4 ? 1 : 2)][dv == 2 ? 0 : (dv == 4 ? 1 : 2)];
    if (!done) {
      if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess)
        return NBLDPC_ERR_CUDA;
      done = true;
    }
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pl.per_sm, k, pl.threads, pl.smem) != cudaSuccess)
    return NBLDPC_ERR_CUDA;
  if (pl.per_sm < 1) return NBLDPC_ERR_UNSUPPORTED;
  pl.grid_max = pl.per_sm * sms;
  pl.slot_bytes = round_up((size_t)c->nnz * c->q * sizeof(float), 256);
  c->fft_plan = pl;
  c->fft_dc = dc;
  c->fft_dv = dv;
  return NBLDPC_OK;
}

namespace {

int fft_launch(const nbldpc_code* c, const float* prob, int frames, int max_iters, int early_stop, uint8_t* sym,
               int32_t* iters, uint8_t* ok, float* app, void* ws, cudaStream_t st) {
  const Plan& pl = c->fft_plan;
  nbldpc::FftParams fp{};
  fp.job.blob = c->blob_dev;
  fp.job.off = c->off;
  fp.job.prob = prob;
  fp.job.out_sym = sym;
  fp.job.out_iters = iters;
  fp.job.out_ok = ok;
  fp.job.out_app = app;
  fp.job.q = c->q;
  fp.job.n = c->n;
  fp.job.m = c->m;
  fp.job.frames = frames;
  fp.job.max_iters = max_iters;
  fp.job.early_stop = early_stop ? 1 : 0;
  fp.counter = reinterpret_cast<unsigned int*>(ws);
  fp.msg = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(ws) + 256);
  fp.slot_floats = pl.slot_bytes / sizeof(float);
  fp.blob_cap = pl.blob_cap;
  fp.n_cap = pl.n_cap;
  fp.w_off = (int)round_up((size_t)(pl.blob_cap + pl.n_cap + 16), 256);
  fp.job.ntasks = c->ntasks;
  cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return NBLDPC_ERR_CUDA;
  void* args[] = {&fp};
  e = cudaLaunchKernel(fft_kernel_for(c->q, c->fft_dc, c->fft_dv), dim3(grid_for(pl, frames)), dim3(pl.threads),
                       args, (size_t)pl.smem, st);
  if (e != cudaSuccess) return NBLDPC_ERR_CUDA;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return NBLDPC_OK;
}

}  // namespace

extern "C" {

// ---- FFT-SPA decoding ----------------------------------------------------------
int nbldpc_fftspa_workspace_size(const nbldpc_code* c, int frames, size_t* bytes) {
  if (!c || frames < 0 || !bytes) return NBLDPC_ERR_ARG;
  if (c->fft_status != NBLDPC_OK) return c->fft_status;
  *bytes = ws_bytes(c->fft_plan, frames);
  return NBLDPC_OK;
}

int nbldpc_fftspa_decode(const nbldpc_code* c, const float* prob_dev, int frames, int max_iters, int early_stop,
                         uint8_t* out_sym_dev, int32_t* out_iters_dev, uint8_t* out_ok_dev, float* out_app_dev,
                         void* workspace_dev, size_t workspace_bytes, void* cuda_stream) {
  if (!c || frames < 0 || max_iters < 0) return NBLDPC_ERR_ARG;
  if (c->fft_status != NBLDPC_OK) return c->fft_status;
  if (frames == 0) return NBLDPC_OK;
  if (!prob_dev || !out_sym_dev || !out_iters_dev || !out_ok_dev || !workspace_dev) return NBLDPC_ERR_ARG;
  if (!aligned(prob_dev, 16) || !aligned(out_iters_dev, 4) || !aligned(workspace_dev, 16)) return NBLDPC_ERR_ARG;
  if (out_app_dev && !aligned(out_app_dev, 16)) return NBLDPC_ERR_ARG;
  if (workspace_bytes < ws_bytes(c->fft_plan, frames)) return NBLDPC_ERR_ARG;
  int st = check_device(c);
  if (st != NBLDPC_OK) return st;
  st = cuda_status(cudaGetLastError());
  if (st != NBLDPC_OK) return st;
  return fft_launch(c, prob_dev, frames, max_iters, early_stop, out_sym_dev, out_iters_dev, out_ok_dev, out_app_dev,
                    workspace_dev, reinterpret_cast<cudaStream_t>(cuda_stream));
}

int nbldpc_fftspa_decode_host_workspace_size(const nbldpc_code* c, int chunk_frames, size_t* bytes) {
  if (!c || !bytes || chunk_frames <= 0) return NBLDPC_ERR_ARG;
  if (c->fft_status != NBLDPC_OK) return c->fft_status;
  *bytes = 2 * host_chunk_bytes(c, chunk_frames, (size_t)c->n * c->q * sizeof(float),
                                ws_bytes(c->fft_plan, chunk_frames));
  return NBLDPC_OK;
}

int nbldpc_fftspa_decode_host(const nbldpc_code* cc, const float* prob_host, int frames, int max_iters,
                              int early_stop, uint8_t* out_sym_host, int32_t* out_iters_host, uint8_t* out_ok_host,
                              int chunk_frames, void* workspace_dev, size_t workspace_bytes, void* cuda_stream) {
  nbldpc_code* c = const_cast<nbldpc_code*>(cc);
  if (!c || frames < 0 || max_iters < 0 || chunk_frames <= 0) return NBLDPC_ERR_ARG;
  if (c->fft_status != NBLDPC_OK) return c->fft_status;
  if (frames == 0) return NBLDPC_OK;
  const int st = check_device(c);
  if (st != NBLDPC_OK) return st;
  const size_t fbytes = (size_t)c->n * c->q * sizeof(float);
  const size_t per = host_chunk_bytes(c, chunk_frames, fbytes, ws_bytes(c->fft_plan, chunk_frames));
  return host_chunks(c, prob_host, fbytes, frames, out_sym_host, out_iters_host, out_ok_host, chunk_frames,
                     workspace_dev, workspace_bytes, per, cuda_stream,
                     [&](const void* in, int nf, uint8_t* sy, int32_t* it, uint8_t* okb, void* ws, cudaStream_t s) {
                       return fft_launch(c, reinterpret_cast<const float*>(in), nf, max_iters, early_stop, sy, it, okb,
                                         nullptr, ws, s);
                     });
}

}  // extern "C"
