// C ABI of the GB300 min-max NB-LDPC decoder (declarations and contracts in
// include/nbldpc.h).  Host side: argument validation, GF tables, code upload,
// launch configuration and stream-ordered launches of the decode kernel.
#include "nbldpc.h"

#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "mma_kernels.cuh"

namespace {

std::atomic<uint64_t> g_launches{0};

struct LaunchCfg {
  int threads = 0;
  int smem = 0;
  int blocks_per_sm = 0;
  int grid_max = 0;
  int group_bytes = 0;
};

}  // namespace

struct nbldpc_code {
  int q = 0, p = 0, n = 0, m = 0, nnz = 0, dmax = 0, vmax = 0;
  uint32_t poly = 0;
  int device = 0;
  unsigned char* blob_dev = nullptr;
  nbldpc::CodeBlob off{};
  LaunchCfg cfg{};
  std::mutex mu;                       // guards the lazily created copy stream
  cudaStream_t side = nullptr;         // second stream for nbldpc_decode_host
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
};

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? NBLDPC_OK : NBLDPC_ERR_CUDA; }

// Field tables by repeated multiplication by x modulo the primitive
// polynomial; fails unless x generates all q-1 non-zero elements.
bool build_field(int q, uint32_t poly, std::vector<uint8_t>& exp2, std::vector<uint8_t>& lg) {
  int p = 0;
  while ((1 << p) < q) ++p;
  if ((poly >> p) != 1u) return false;
  exp2.assign(2 * q, 0);
  lg.assign(q, 0);
  std::vector<int> seen(q, 0);
  uint32_t v = 1;
  for (int i = 0; i < q - 1; ++i) {
    if (seen[v]) return false;
    seen[v] = 1;
    exp2[i] = (uint8_t)v;
    lg[v] = (uint8_t)i;
    v <<= 1;
    if (v & (uint32_t)q) v ^= poly;
  }
  if (v != 1u) return false;
  for (int i = q - 1; i < 2 * q; ++i) exp2[i] = exp2[i % (q - 1)];
  return true;
}

template <int Q> const void* kernel_ptr() { return reinterpret_cast<const void*>(&nbldpc::mma_decode_kernel<Q>); }

const void* kernel_for(int q) {
  switch (q) {
    case 2: return kernel_ptr<2>();
    case 4: return kernel_ptr<4>();
    case 8: return kernel_ptr<8>();
    case 16: return kernel_ptr<16>();
    case 32: return kernel_ptr<32>();
    case 64: return kernel_ptr<64>();
    case 128: return kernel_ptr<128>();
    case 256: return kernel_ptr<256>();
  }
  return nullptr;
}

int group_lanes(int q) {
  switch (q) {
    case 2: return nbldpc::Geo<2>::G;
    case 4: return nbldpc::Geo<4>::G;
    case 8: return nbldpc::Geo<8>::G;
    case 16: return nbldpc::Geo<16>::G;
    case 32: return nbldpc::Geo<32>::G;
    case 64: return nbldpc::Geo<64>::G;
    case 128: return nbldpc::Geo<128>::G;
    case 256: return nbldpc::Geo<256>::G;
  }
  return 0;
}

int scratch_bytes(int q, int dmax) {
  switch (q) {
    case 2: return nbldpc::group_scratch_bytes<2>(dmax);
    case 4: return nbldpc::group_scratch_bytes<4>(dmax);
    case 8: return nbldpc::group_scratch_bytes<8>(dmax);
    case 16: return nbldpc::group_scratch_bytes<16>(dmax);
    case 32: return nbldpc::group_scratch_bytes<32>(dmax);
    case 64: return nbldpc::group_scratch_bytes<64>(dmax);
    case 128: return nbldpc::group_scratch_bytes<128>(dmax);
    case 256: return nbldpc::group_scratch_bytes<256>(dmax);
  }
  return 0;
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Block size, shared memory and resident blocks for a code on the current device.
int configure(nbldpc_code* c) {
  int dev = 0, sms = 0, smem_optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return NBLDPC_ERR_CUDA;
  const int G = group_lanes(c->q);
  const int work = (c->m > c->n ? c->m : c->n) * G;
  int threads = (int)round_up((size_t)work, 32);
  if (threads > 256) threads = 256;
  if (threads < 32) threads = 32;
  const int gb = scratch_bytes(c->q, c->dmax);
  const int fixed = c->off.bytes + (int)round_up((size_t)c->n, 16) + 64;
  while (threads > 32 && fixed + (threads / G) * gb > smem_optin) threads -= 32;
  const int smem = fixed + (threads / G) * gb;
  if (smem > smem_optin) return NBLDPC_ERR_UNSUPPORTED;
  const void* k = kernel_for(c->q);
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return NBLDPC_ERR_CUDA;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
  if (e != cudaSuccess) return NBLDPC_ERR_CUDA;
  if (per_sm < 1) return NBLDPC_ERR_UNSUPPORTED;
  c->cfg.threads = threads;
  c->cfg.smem = smem;
  c->cfg.blocks_per_sm = per_sm;
  c->cfg.grid_max = per_sm * sms;
  c->cfg.group_bytes = gb;
  return NBLDPC_OK;
}

size_t slot_bytes(const nbldpc_code* c) { return round_up((size_t)c->nnz * c->q, 256); }

int grid_for(const nbldpc_code* c, int frames) { return frames < c->cfg.grid_max ? frames : c->cfg.grid_max; }

size_t decode_ws_bytes(const nbldpc_code* c, int frames) {
  return 256 + (size_t)grid_for(c, frames) * slot_bytes(c);
}

int launch(const nbldpc_code* c, const uint8_t* gamma, int frames, int max_iters, int early_stop,
           uint8_t* sym, int32_t* iters, uint8_t* ok, void* ws, cudaStream_t st) {
  if (frames == 0) return NBLDPC_OK;
  nbldpc::DecodeParams prm{};
  prm.gamma = gamma;
  prm.out_sym = sym;
  prm.out_iters = iters;
  prm.out_ok = ok;
  prm.counter = reinterpret_cast<unsigned int*>(ws);
  prm.msg = reinterpret_cast<uint8_t*>(ws) + 256;
  prm.blob = c->blob_dev;
  prm.off = c->off;
  prm.slot_bytes = slot_bytes(c);
  prm.n = c->n;
  prm.m = c->m;
  prm.nnz = c->nnz;
  prm.dmax = c->dmax;
  prm.frames = frames;
  prm.max_iters = max_iters;
  prm.early_stop = early_stop ? 1 : 0;
  prm.group_bytes = c->cfg.group_bytes;
  prm.key16 = (255 * (c->vmax + 1) + 1) * c->q <= 65536 ? 1 : 0;
  cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return NBLDPC_ERR_CUDA;
  const int grid = grid_for(c, frames);
  void* args[] = {&prm};
  e = cudaLaunchKernel(kernel_for(c->q), dim3(grid), dim3(c->cfg.threads), args, (size_t)c->cfg.smem, st);
  if (e != cudaSuccess) return NBLDPC_ERR_CUDA;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return NBLDPC_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// ---- non-allocating decode (nbldpc_decode_noalloc) -------------------------
// Fixed scratch for callers that cannot allocate: frame counter + message slots.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NBLDPC_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256] = {};

// Device address of g_noalloc_scratch on the current device (looked up once per
// device, with that device current; host code must not use the symbol itself).
int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return NBLDPC_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return NBLDPC_ERR_CUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return NBLDPC_OK;
}

int launch_noalloc(const nbldpc_code* c, const uint8_t* gamma, int frames, int max_iters, int early_stop,
                   uint8_t* sym, int32_t* iters, uint8_t* ok, void* scratch, int grid, cudaStream_t st) {
  nbldpc::DecodeParams prm{};
  prm.gamma = gamma;
  prm.out_sym = sym;
  prm.out_iters = iters;
  prm.out_ok = ok;
  prm.counter = reinterpret_cast<unsigned int*>(scratch);
  prm.msg = reinterpret_cast<uint8_t*>(scratch) + 256;
  prm.blob = c->blob_dev;
  prm.off = c->off;
  prm.slot_bytes = slot_bytes(c);
  prm.n = c->n;
  prm.m = c->m;
  prm.nnz = c->nnz;
  prm.dmax = c->dmax;
  prm.frames = frames;
  prm.max_iters = max_iters;
  prm.early_stop = early_stop ? 1 : 0;
  prm.group_bytes = c->cfg.group_bytes;
  prm.key16 = (255 * (c->vmax + 1) + 1) * c->q <= 65536 ? 1 : 0;
  // the array keeps the previous call's contents: the frame counter must start at zero
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return NBLDPC_ERR_CUDA;
  void* args[] = {&prm};
  e = cudaLaunchKernel(kernel_for(c->q), dim3(grid), dim3(c->cfg.threads), args, (size_t)c->cfg.smem, st);
  if (e != cudaSuccess) return NBLDPC_ERR_CUDA;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return NBLDPC_OK;
}

}  // namespace

extern "C" {

int nbldpc_decode_noalloc(const nbldpc_code* c, const uint8_t* gamma_dev, int frames, int max_iters,
                          int early_stop, uint8_t* out_sym_dev, int32_t* out_iters_dev, uint8_t* out_ok_dev,
                          void* cuda_stream) {
  if (!c || frames < 0 || max_iters < 0) return NBLDPC_ERR_ARG;
  if (frames == 0) return NBLDPC_OK;
  if (!gamma_dev || !out_sym_dev || !out_iters_dev || !out_ok_dev) return NBLDPC_ERR_ARG;
  if (!aligned(gamma_dev, 16) || !aligned(out_iters_dev, 4)) return NBLDPC_ERR_ARG;
  const size_t slot = slot_bytes(c);
  if (256 + slot > (size_t)NBLDPC_NOALLOC_SCRATCH_BYTES) return NBLDPC_ERR_UNSUPPORTED;
  const int fit = (int)(((size_t)NBLDPC_NOALLOC_SCRATCH_BYTES - 256) / slot);
  int grid = grid_for(c, frames);
  if (grid > fit) grid = fit;
  int st = cuda_status(cudaGetLastError());
  if (st != NBLDPC_OK) return st;
  void* scratch = nullptr;
  st = noalloc_scratch(&scratch);
  if (st != NBLDPC_OK) return st;
  return launch_noalloc(c, gamma_dev, frames, max_iters, early_stop, out_sym_dev, out_iters_dev, out_ok_dev,
                        scratch, grid, reinterpret_cast<cudaStream_t>(cuda_stream));
}

const char* nbldpc_status_string(int status) {
  switch (status) {
    case NBLDPC_OK: return "ok";
    case NBLDPC_ERR_ARG: return "invalid argument";
    case NBLDPC_ERR_POLY: return "field order not a power of two in [2,256] or polynomial not primitive";
    case NBLDPC_ERR_H: return "malformed parity-check matrix";
    case NBLDPC_ERR_CUDA: return "CUDA error";
    case NBLDPC_ERR_NOMEM: return "out of memory";
    case NBLDPC_ERR_TIMEOUT: return "device-side wait timed out";
    case NBLDPC_ERR_UNSUPPORTED: return "code outside the supported limits";
  }
  return "unknown status";
}

uint64_t nbldpc_kernel_launch_count(void) { return g_launches.load(); }

int nbldpc_code_create(int q, uint32_t prim_poly, int n_cols, int n_rows, const int32_t* row_ptr,
                       const int32_t* col_idx, const uint8_t* coef, nbldpc_code** out) {
  if (!out) return NBLDPC_ERR_ARG;
  *out = nullptr;
  if (!row_ptr || !col_idx || !coef || n_cols <= 0 || n_rows <= 0) return NBLDPC_ERR_ARG;
  if (q < 2 || q > 256 || (q & (q - 1))) return NBLDPC_ERR_POLY;
  std::vector<uint8_t> exp2, lg;
  if (!build_field(q, prim_poly, exp2, lg)) return NBLDPC_ERR_POLY;
  if (row_ptr[0] != 0) return NBLDPC_ERR_H;
  for (int r = 0; r < n_rows; ++r)
    if (row_ptr[r + 1] - row_ptr[r] < 2) return NBLDPC_ERR_H;
  const int64_t nnz64 = row_ptr[n_rows];
  if (n_cols >= 65535 || nnz64 >= 65535) return NBLDPC_ERR_UNSUPPORTED;
  const int nnz = (int)nnz64;
  std::vector<int> vdeg(n_cols, 0), last(n_cols, -1);
  int dmax = 0;
  for (int r = 0; r < n_rows; ++r) {
    const int d = row_ptr[r + 1] - row_ptr[r];
    if (d > dmax) dmax = d;
    for (int e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
      const int c = col_idx[e];
      if (c < 0 || c >= n_cols || coef[e] == 0 || coef[e] >= q || last[c] == r) return NBLDPC_ERR_H;
      last[c] = r;
      ++vdeg[c];
    }
  }
  int vmax = 0;
  for (int c = 0; c < n_cols; ++c) {
    if (vdeg[c] < 1) return NBLDPC_ERR_H;
    if (vdeg[c] > vmax) vmax = vdeg[c];
  }
  if (dmax > 64 || vmax > 64) return NBLDPC_ERR_UNSUPPORTED;

  // code blob: exp2 | log | row_ptr u16 | edge_col u16 | edge_lh u8 | edge_lhi u8 | vn_ptr u16 | vn_edge u16
  nbldpc::CodeBlob off{};
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = o; o = round_up(o + bytes, 16); return (int)at; };
  off.exp2 = take(2 * (size_t)q);
  off.log = take((size_t)q);
  off.row_ptr = take(2 * ((size_t)n_rows + 1));
  off.edge_col = take(2 * (size_t)nnz);
  off.edge_lh = take((size_t)nnz);
  off.edge_lhi = take((size_t)nnz);
  off.vn_ptr = take(2 * ((size_t)n_cols + 1));
  off.vn_edge = take(2 * (size_t)nnz);
  off.bytes = (int)o;
  std::vector<unsigned char> blob(o, 0);
  memcpy(&blob[off.exp2], exp2.data(), 2 * (size_t)q);
  memcpy(&blob[off.log], lg.data(), (size_t)q);
  uint16_t* rp = reinterpret_cast<uint16_t*>(&blob[off.row_ptr]);
  uint16_t* ec = reinterpret_cast<uint16_t*>(&blob[off.edge_col]);
  uint8_t* elh = &blob[off.edge_lh];
  uint8_t* elhi = &blob[off.edge_lhi];
  uint16_t* vp = reinterpret_cast<uint16_t*>(&blob[off.vn_ptr]);
  uint16_t* ve = reinterpret_cast<uint16_t*>(&blob[off.vn_edge]);
  for (int r = 0; r <= n_rows; ++r) rp[r] = (uint16_t)row_ptr[r];
  for (int e = 0; e < nnz; ++e) {
    ec[e] = (uint16_t)col_idx[e];
    elh[e] = lg[coef[e]];
    elhi[e] = (uint8_t)((q - 1 - lg[coef[e]]) % (q - 1));
  }
  vp[0] = 0;
  for (int c = 0; c < n_cols; ++c) vp[c + 1] = (uint16_t)(vp[c] + vdeg[c]);
  std::vector<int> fill(n_cols, 0);
  for (int e = 0; e < nnz; ++e) {
    const int c = col_idx[e];
    ve[vp[c] + fill[c]++] = (uint16_t)e;
  }

  nbldpc_code* c = new (std::nothrow) nbldpc_code();
  if (!c) return NBLDPC_ERR_NOMEM;
  c->q = q;
  c->p = 0;
  while ((1 << c->p) < q) ++c->p;
  c->n = n_cols;
  c->m = n_rows;
  c->nnz = nnz;
  c->dmax = dmax;
  c->vmax = vmax;
  c->poly = prim_poly;
  c->off = off;
  if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return NBLDPC_ERR_CUDA; }
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&c->blob_dev), o);
  if (e != cudaSuccess) { delete c; return e == cudaErrorMemoryAllocation ? NBLDPC_ERR_NOMEM : NBLDPC_ERR_CUDA; }
  e = cudaMemcpy(c->blob_dev, blob.data(), o, cudaMemcpyHostToDevice);
  int st = cuda_status(e);
  if (st == NBLDPC_OK) st = configure(c);
  if (st != NBLDPC_OK) {
    cudaFree(c->blob_dev);
    delete c;
    return st;
  }
  *out = c;
  return NBLDPC_OK;
}

void nbldpc_code_destroy(nbldpc_code* c) {
  if (!c) return;
  for (auto& ev : c->ev)
    if (ev) cudaEventDestroy(ev);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->blob_dev) cudaFree(c->blob_dev);
  delete c;
}

int nbldpc_code_info(const nbldpc_code* c, int* q, int* n, int* m, int* nnz) {
  if (!c) return NBLDPC_ERR_ARG;
  if (q) *q = c->q;
  if (n) *n = c->n;
  if (m) *m = c->m;
  if (nnz) *nnz = c->nnz;
  return NBLDPC_OK;
}

int nbldpc_decode_workspace_size(const nbldpc_code* c, int frames, size_t* bytes) {
  if (!c || !bytes || frames < 0) return NBLDPC_ERR_ARG;
  *bytes = decode_ws_bytes(c, frames);
  return NBLDPC_OK;
}

int nbldpc_decode(const nbldpc_code* c, const uint8_t* gamma_dev, int frames, int max_iters, int early_stop,
                  uint8_t* out_sym_dev, int32_t* out_iters_dev, uint8_t* out_ok_dev, void* workspace_dev,
                  size_t workspace_bytes, void* cuda_stream) {
  if (!c || frames < 0 || max_iters < 0) return NBLDPC_ERR_ARG;
  if (frames == 0) return NBLDPC_OK;
  if (!gamma_dev || !out_sym_dev || !out_iters_dev || !out_ok_dev || !workspace_dev) return NBLDPC_ERR_ARG;
  if (!aligned(gamma_dev, 16) || !aligned(workspace_dev, 16) || !aligned(out_iters_dev, 4)) return NBLDPC_ERR_ARG;
  if (workspace_bytes < decode_ws_bytes(c, frames)) return NBLDPC_ERR_ARG;
  int st = cuda_status(cudaGetLastError());
  if (st != NBLDPC_OK) return st;
  return launch(c, gamma_dev, frames, max_iters, early_stop, out_sym_dev, out_iters_dev, out_ok_dev,
                workspace_dev, reinterpret_cast<cudaStream_t>(cuda_stream));
}

int nbldpc_decode_host_workspace_size(const nbldpc_code* c, int chunk_frames, size_t* bytes) {
  if (!c || !bytes || chunk_frames <= 0) return NBLDPC_ERR_ARG;
  const size_t per = round_up((size_t)chunk_frames * c->n * c->q, 256) + round_up((size_t)chunk_frames * c->n, 256) +
                     round_up((size_t)chunk_frames * 4, 256) + round_up((size_t)chunk_frames, 256) +
                     round_up(decode_ws_bytes(c, chunk_frames), 256);
  *bytes = 2 * per;
  return NBLDPC_OK;
}

int nbldpc_decode_host(const nbldpc_code* cc, const uint8_t* gamma_host, int frames, int max_iters, int early_stop,
                       uint8_t* out_sym_host, int32_t* out_iters_host, uint8_t* out_ok_host, int chunk_frames,
                       void* workspace_dev, size_t workspace_bytes, void* cuda_stream) {
  nbldpc_code* c = const_cast<nbldpc_code*>(cc);
  if (!c || frames < 0 || max_iters < 0 || chunk_frames <= 0) return NBLDPC_ERR_ARG;
  if (frames == 0) return NBLDPC_OK;
  if (!gamma_host || !out_sym_host || !out_iters_host || !out_ok_host || !workspace_dev) return NBLDPC_ERR_ARG;
  if (!aligned(workspace_dev, 256)) return NBLDPC_ERR_ARG;
  size_t need = 0;
  nbldpc_decode_host_workspace_size(c, chunk_frames, &need);
  if (workspace_bytes < need) return NBLDPC_ERR_ARG;
  int st = cuda_status(cudaGetLastError());
  if (st != NBLDPC_OK) return st;
  cudaStream_t main = reinterpret_cast<cudaStream_t>(cuda_stream);
  {
    std::lock_guard<std::mutex> lk(c->mu);
    if (!c->side) {
      if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess) return NBLDPC_ERR_CUDA;
      for (auto& ev : c->ev)
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return NBLDPC_ERR_CUDA;
    }
  }
  std::lock_guard<std::mutex> lk(c->mu);  // one host decode at a time per handle (shared side stream)
  const size_t g_b = round_up((size_t)chunk_frames * c->n * c->q, 256), s_b = round_up((size_t)chunk_frames * c->n, 256),
               i_b = round_up((size_t)chunk_frames * 4, 256), o_b = round_up((size_t)chunk_frames, 256);
  const size_t per = need / 2;
  cudaStream_t streams[2] = {main, c->side};
  // the side stream starts after work already queued on the caller's stream
  if (cudaEventRecord(c->ev[0], main) != cudaSuccess || cudaStreamWaitEvent(c->side, c->ev[0], 0) != cudaSuccess)
    return NBLDPC_ERR_CUDA;
  const size_t fbytes = (size_t)c->n * c->q;
  for (int f0 = 0, i = 0; f0 < frames; f0 += chunk_frames, ++i) {
    const int nf = frames - f0 < chunk_frames ? frames - f0 : chunk_frames;
    unsigned char* base = reinterpret_cast<unsigned char*>(workspace_dev) + (size_t)(i & 1) * per;
    uint8_t* g = base;
    uint8_t* sy = base + g_b;
    int32_t* it = reinterpret_cast<int32_t*>(base + g_b + s_b);
    uint8_t* okb = base + g_b + s_b + i_b;
    void* ws = base + g_b + s_b + i_b + o_b;
    cudaStream_t s = streams[i & 1];
    cudaError_t e = cudaMemcpyAsync(g, gamma_host + (size_t)f0 * fbytes, (size_t)nf * fbytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return NBLDPC_ERR_CUDA;
    st = launch(c, g, nf, max_iters, early_stop, sy, it, okb, ws, s);
    if (st != NBLDPC_OK) return st;
    e = cudaMemcpyAsync(out_sym_host + (size_t)f0 * c->n, sy, (size_t)nf * c->n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_iters_host + f0, it, (size_t)nf * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_ok_host + f0, okb, (size_t)nf, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return NBLDPC_ERR_CUDA;
  }
  // the caller's stream completes only after the side stream's chunks
  if (cudaEventRecord(c->ev[1], c->side) != cudaSuccess || cudaStreamWaitEvent(main, c->ev[1], 0) != cudaSuccess)
    return NBLDPC_ERR_CUDA;
  return NBLDPC_OK;
}

}  // extern "C"
