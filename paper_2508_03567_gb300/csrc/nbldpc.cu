// C ABI of the GB300 NB-LDPC decoders (declarations and contracts in
// include/nbldpc.h), min-max side: argument validation, GF tables, code upload
// (with the FFT-SPA blob section), launch planning, mixed batches, the
// autotuner, host-buffer and non-allocating decodes, stream-ordered launches
// of the min-max kernels.  FFT-SPA decodes are in fftspa_host.cu.
#include "nbldpc.h"

#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "host_internal.h"
#include "mma_kernels.cuh"

static_assert(nbldpc::kMaxJobs == NBLDPC_MAX_BATCH_JOBS, "job table size");
static_assert(sizeof(nbldpc::LaunchParams) < 32000, "kernel parameter space");

std::atomic<uint64_t> nbldpc_host::g_launches{0};
std::mutex nbldpc_host::g_attr_mu;

using namespace nbldpc_host;

namespace {

constexpr int kThreads = 256;

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

}  // namespace

namespace nbldpc {   // defined in kernels.cu, one translation unit per field order
const void* kernel_q0(int v, int mb, int t1, int dreg);
const void* kernel_q2(int v, int mb, int t1, int dreg);
const void* kernel_q4(int v, int mb, int t1, int dreg);
const void* kernel_q8(int v, int mb, int t1, int dreg);
const void* kernel_q16(int v, int mb, int t1, int dreg);
const void* kernel_q32(int v, int mb, int t1, int dreg);
const void* kernel_q64(int v, int mb, int t1, int dreg);
const void* kernel_q128(int v, int mb, int t1, int dreg);
const void* kernel_q256(int v, int mb, int t1, int dreg);
}  // namespace nbldpc

namespace {

// Kernel mode: 1 = 8-bit messages, 2 = 16-bit messages, 3 = 8-bit messages with
// the Table 1 check-node schedule (each a separate kernel instantiation).
int kmode(const nbldpc_code* c) { return c->mb == 2 ? 2 : (c->cnp_schedule == NBLDPC_CNP_TABLE1 ? 3 : 1); }

// kernel compiled for one field order, variant (bit 0: layout; bit 1: messages
// resident in shared memory; bit 2: pruned convolutions), kernel mode and the
// code's regular check degree (dreg: 0 when the rows differ; a field order may
// have a kernel for it), or for every field order (q = 0, mode 1)
const void* kernel_for(int q, int v, int km, int dreg = 0) {
  const int mb = km == 2 ? 2 : 1, t1 = km == 3 ? 1 : 0;
  switch (q) {
    case 0: return nbldpc::kernel_q0(-1, mb, t1, 0);
    case 2: return nbldpc::kernel_q2(v, mb, t1, dreg);
    case 4: return nbldpc::kernel_q4(v, mb, t1, dreg);
    case 8: return nbldpc::kernel_q8(v, mb, t1, dreg);
    case 16: return nbldpc::kernel_q16(v, mb, t1, dreg);
    case 32: return nbldpc::kernel_q32(v, mb, t1, dreg);
    case 64: return nbldpc::kernel_q64(v, mb, t1, dreg);
    case 128: return nbldpc::kernel_q128(v, mb, t1, dreg);
    case 256: return nbldpc::kernel_q256(v, mb, t1, dreg);
  }
  return nullptr;
}

// the regular check degree that selects a specialised kernel (see kernel_for), else 0
int kernel_dreg(int q, int v, int km, int dreg) {
  return ((q == 64 || q == 4) && km == 1 && v >= 2 && v <= 3 && dreg == 4) ? 4 : 0;
}

template <int Q> int lanes(int v) { return v ? nbldpc::Geo<Q, 1>::G : nbldpc::Geo<Q, 0>::G; }

int group_lanes(int q, int v) {
  switch (q) {
    case 2: return lanes<2>(v);
    case 4: return lanes<4>(v);
    case 8: return lanes<8>(v);
    case 16: return lanes<16>(v);
    case 32: return lanes<32>(v);
    case 64: return lanes<64>(v);
    case 128: return lanes<128>(v);
    case 256: return lanes<256>(v);
  }
  return 0;
}

int group_bytes(int q, int dmax, int mb) {
  switch (q) {
    case 2: return nbldpc::group_scratch_bytes<2>(dmax, mb);
    case 4: return nbldpc::group_scratch_bytes<4>(dmax, mb);
    case 8: return nbldpc::group_scratch_bytes<8>(dmax, mb);
    case 16: return nbldpc::group_scratch_bytes<16>(dmax, mb);
    case 32: return nbldpc::group_scratch_bytes<32>(dmax, mb);
    case 64: return nbldpc::group_scratch_bytes<64>(dmax, mb);
    case 128: return nbldpc::group_scratch_bytes<128>(dmax, mb);
    case 256: return nbldpc::group_scratch_bytes<256>(dmax, mb);
  }
  return 0;
}

// Every kernel may use up to the opt-in shared memory of the device (set once
// per device and kernel; occupancy still follows the bytes of each launch).
bool g_attr_done[64][85] = {};

// per field order: 3 kernel modes x 2 layouts, the 2 resident-message kernels,
// then the 2 pruned-convolution kernels; after them the 2 GF(64) and the 2 GF(4)
// resident kernels of check degree 4
int kernel_slot(int q, int v, int km, int dreg) {
  if (q == 0) return 0;
  if (kernel_dreg(q, v, km, dreg)) return (q == 64 ? 81 : 83) + (v & 1);
  return 1 + 10 * (nbldpc::ilog2(q) - 1) + ((v & 4) ? 8 + (v & 1) : (v & 2) ? 6 + (v & 1) : 2 * (km - 1) + (v & 1));
}

int prepare_kernel(int q, int v, int km, int dreg, int dev, int smem_optin) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (dev < 0 || dev >= 64) return NBLDPC_ERR_CUDA;
  const void* k = kernel_for(q, v, km, dreg);
  if (!k) return NBLDPC_ERR_UNSUPPORTED;
  bool& done = g_attr_done[dev][kernel_slot(q, v, km, dreg)];
  if (!done) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin) != cudaSuccess)
      return NBLDPC_ERR_CUDA;
    done = true;
  }
  return NBLDPC_OK;
}

struct CodeNeeds {       // what one code asks of a frame slot
  int q, variant, mb, dmax, blob, n;
  size_t msg;
  int dreg;              // regular check degree (0: the rows differ)
};

CodeNeeds needs_of(const nbldpc_code* c, int variant, int mb) {
  return CodeNeeds{c->q, variant, mb, c->dmax, c->off.bytes, c->n, round_up((size_t)c->nnz * c->q * mb, 256),
                   c->dreg};
}

// Plan a launch of kernel (kq, kv, kernel mode km) with fpb frame slots per block for a set of codes.
// Variants 2 and 3 keep each frame's messages in shared memory: blocks of
// nbldpc::kResidentThreads threads (1, 2 or 4 frame slots) or of 256 threads with
// 8 one-warp slots, no message slots in the workspace.
int make_plan(int kq, int kv, int km, int fpb, const CodeNeeds* cs, int nc, Plan* out) {
  int dev = 0, sms = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return NBLDPC_ERR_CUDA;
  const bool resident = kv >= 0 && (kv & 2);
  const int threads = resident ? (fpb == 8 ? kThreads : nbldpc::kResidentThreads) : kThreads;
  if (fpb < 1 || threads % fpb) return NBLDPC_ERR_ARG;
  if (resident && km != 1) return NBLDPC_ERR_UNSUPPORTED;
  const int nthr = threads / fpb;
  if (nthr < 32 || nthr % 32) return NBLDPC_ERR_UNSUPPORTED;
  Plan pl{};
  pl.fpb = fpb;
  pl.threads = threads;
  int scratch = 0;
  for (int i = 0; i < nc; ++i) {
    const int G = group_lanes(cs[i].q, cs[i].variant & 1);
    if (G > nthr) return NBLDPC_ERR_UNSUPPORTED;
    const int s = (nthr / G) * group_bytes(cs[i].q, cs[i].dmax, cs[i].mb);
    if (s > scratch) scratch = s;
    if (cs[i].blob > pl.blob_cap) pl.blob_cap = cs[i].blob;
    if (cs[i].n > pl.n_cap) pl.n_cap = cs[i].n;
    if (cs[i].msg > pl.slot_bytes) pl.slot_bytes = cs[i].msg;
  }
  pl.blob_cap = (int)round_up((size_t)pl.blob_cap, 16);
  pl.n_cap = (int)round_up((size_t)pl.n_cap, 16);
  pl.slot_smem = (int)round_up((size_t)(pl.blob_cap + pl.n_cap + 16 + scratch), 16);
  if (resident) {   // the messages follow the slot's scratch
    pl.xs_off = pl.slot_smem;
    pl.slot_smem += (int)round_up(pl.slot_bytes, 16);
    pl.slot_bytes = 0;
  }
  pl.smem = fpb * pl.slot_smem;
  if (pl.smem > optin) return NBLDPC_ERR_UNSUPPORTED;
  const int dreg = (kq != 0 && nc == 1) ? cs[0].dreg : 0;
  int st = prepare_kernel(kq, kv, km, dreg, dev, optin);
  if (st != NBLDPC_OK) return st;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pl.per_sm, kernel_for(kq, kv, km, dreg), pl.threads, pl.smem) !=
      cudaSuccess)
    return NBLDPC_ERR_CUDA;
  if (pl.per_sm < 1) return NBLDPC_ERR_UNSUPPORTED;
  pl.grid_max = pl.per_sm * sms;
  *out = pl;
  return NBLDPC_OK;
}

// Variant when nothing better is known: the one measured fastest for the
// benchmark codes on GB300 (GF(16), GF(32): layout 1; GF(64): layout 1 with
// the messages in shared memory; GF(4): layout 0 with the messages in shared
// memory; GF(128), GF(256): pruned convolutions, layout 0 (GF(256) (2,6) N=384:
// 2.8x the dense kernel; GF(128) (2,4) N=256: 35.6 against 41.1 ms); otherwise
// layout 0).
int default_variant(int q) { return q >= 128 ? 4 : q == 64 ? 3 : q == 4 ? 2 : (q >= 16 && q <= 32) ? 1 : 0; }

// GF(4) codes a single warp decodes alone (one-warp frame slots: at most 32
// checks of degree <= 4, columns of degree <= 2): GF(4) N=48 (2,4) 17-18 us per
// 1,000-frame decode at 8 frames per block against 24.5 at 4.
bool warp4_code(const nbldpc_code* c) { return c->q == 4 && c->m <= 32 && c->dmax <= 4 && c->vmax <= 2; }

// Frame slots per block when nothing better is known: enough threads per slot
// for the checks and variable nodes of one frame, at least one warp.
int default_fpb(const nbldpc_code* c) {
  if (warp4_code(c)) return 8;
  const int G = group_lanes(c->q, default_variant(c->q) & 1);
  const int work = c->m * G;
  int fpb = 1;
  while (fpb < 8 && kThreads / (2 * fpb) >= 32 && kThreads / (2 * fpb) >= work && kThreads / (2 * fpb) >= G) fpb *= 2;
  return fpb;
}

int configure(nbldpc_code* c, int variant, int fpb) {
  Plan pl{};
  const CodeNeeds need = needs_of(c, variant, c->mb);
  const int st = make_plan(c->q, variant, kmode(c), fpb, &need, 1, &pl);
  if (st != NBLDPC_OK) return st;
  c->variant = variant;
  c->plan = pl;
  return NBLDPC_OK;
}

size_t decode_ws_bytes(const nbldpc_code* c, int frames) { return ws_bytes(c->plan, frames); }

nbldpc::JobDesc job_desc(const nbldpc_code* c, const uint8_t* gamma, int frames, int max_iters, int early_stop,
                         uint8_t* sym, int32_t* iters, uint8_t* ok, int item_begin, bool count = true) {
  nbldpc::JobDesc j{};
  j.blob = c->blob_dev;
  j.off = c->off;
  j.gamma = gamma;
  j.out_sym = sym;
  j.out_iters = iters;
  j.out_ok = ok;
  j.q = c->q;
  j.n = c->n;
  j.m = c->m;
  j.dmax = c->dmax;
  j.variant = c->variant & 5;          // layout and pruning (a mixed-code kernel keeps messages in the workspace)
  j.work = count ? c->work_counter : nullptr;
  j.vmax = c->vmax;
  j.key16 = (255 * (c->vmax + 1) + 1) * c->q <= 65536 ? 1 : 0;
  j.group_bytes = group_bytes(c->q, c->dmax, c->mb);
  j.frames = frames;
  j.max_iters = max_iters;
  j.early_stop = early_stop ? 1 : 0;
  j.item_begin = item_begin;
  return j;
}

// Queue the counter reset (not needed when every frame has its own slot) and the
// persistent kernel (grid blocks) on st.
int launch_plan(const void* kernel, const Plan& pl, nbldpc::LaunchParams& lp, int grid, void* counter, uint8_t* msg,
                cudaStream_t st) {
  if (lp.total_items == 0 || grid < 1) return NBLDPC_OK;
  lp.counter = reinterpret_cast<unsigned int*>(counter);
  lp.msg = msg;
  lp.slot_bytes = pl.slot_bytes;
  lp.fpb = pl.fpb;
  lp.slot_smem = pl.slot_smem;
  lp.blob_cap = pl.blob_cap;
  lp.n_cap = pl.n_cap;
  lp.xs_off = pl.xs_off;
  // no more frames than frame slots: slot s takes frame s, no counter to reset
  lp.static_items = (long long)lp.total_items <= (long long)grid * pl.fpb ? 1 : 0;
  cudaError_t e = cudaSuccess;
  if (!lp.static_items) {
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return NBLDPC_ERR_CUDA;
  }
  void* args[] = {&lp};
  e = cudaLaunchKernel(kernel, dim3(grid), dim3(pl.threads), args, (size_t)pl.smem, st);
  if (e != cudaSuccess) return NBLDPC_ERR_CUDA;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return NBLDPC_OK;
}

int launch(const nbldpc_code* c, const uint8_t* gamma, int frames, int max_iters, int early_stop, uint8_t* sym,
           int32_t* iters, uint8_t* ok, void* ws, cudaStream_t st, bool count = true) {
  if (frames == 0) return NBLDPC_OK;
  nbldpc::LaunchParams lp{};
  lp.jobs[0] = job_desc(c, gamma, frames, max_iters, early_stop, sym, iters, ok, 0, count);
  lp.njobs = 1;
  lp.total_items = frames;
  return launch_plan(kernel_for(c->q, c->variant, kmode(c), c->dreg), c->plan, lp, grid_for(c->plan, frames), ws,
                     reinterpret_cast<uint8_t*>(ws) + 256, st);
}

// ---- non-allocating decode (nbldpc_decode_noalloc) -------------------------
// Fixed scratch for callers that cannot allocate: frame counter + message slots.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NBLDPC_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch in the current device's context.  Looked
// up on every call (a cheap table lookup once the module is loaded), so the
// address stays right after a context is torn down and re-created; host code
// must not use the symbol itself, which names a host-side stand-in.
int noalloc_scratch(void** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return NBLDPC_ERR_CUDA;
  *out = p;
  return NBLDPC_OK;
}

bool valid_outputs(const uint8_t* gamma, const uint8_t* sym, const int32_t* iters, const uint8_t* ok) {
  return gamma && sym && iters && ok && aligned(gamma, 16) && aligned(iters, 4);
}

}  // namespace

extern "C" {

int nbldpc_decode_noalloc(const nbldpc_code* c, const uint8_t* gamma_dev, int frames, int max_iters,
                          int early_stop, uint8_t* out_sym_dev, int32_t* out_iters_dev, uint8_t* out_ok_dev,
                          void* cuda_stream) {
  if (!c || frames < 0 || max_iters < 0) return NBLDPC_ERR_ARG;
  if (frames == 0) return NBLDPC_OK;
  if (!valid_outputs(gamma_dev, out_sym_dev, out_iters_dev, out_ok_dev)) return NBLDPC_ERR_ARG;
  int st = check_device(c);
  if (st != NBLDPC_OK) return st;
  const Plan& pl = c->plan;
  const size_t per_block = (size_t)pl.fpb * pl.slot_bytes;   // 0 when the messages stay in shared memory
  if (256 + per_block > (size_t)NBLDPC_NOALLOC_SCRATCH_BYTES) return NBLDPC_ERR_UNSUPPORTED;
  int grid = grid_for(pl, frames);
  if (per_block) {
    const int fit = (int)(((size_t)NBLDPC_NOALLOC_SCRATCH_BYTES - 256) / per_block);
    if (grid > fit) grid = fit;
  }
  st = cuda_status(cudaGetLastError());
  if (st != NBLDPC_OK) return st;
  void* scratch = nullptr;
  st = noalloc_scratch(&scratch);
  if (st != NBLDPC_OK) return st;
  // the array keeps the previous call's contents: the frame counter is cleared in launch_plan
  nbldpc::LaunchParams lp{};
  lp.jobs[0] = job_desc(c, gamma_dev, frames, max_iters, early_stop, out_sym_dev, out_iters_dev, out_ok_dev, 0);
  lp.njobs = 1;
  lp.total_items = frames;
  return launch_plan(kernel_for(c->q, c->variant, kmode(c), c->dreg), pl, lp, grid, scratch,
                     reinterpret_cast<uint8_t*>(scratch) + 256,
                     reinterpret_cast<cudaStream_t>(cuda_stream));
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
  // FFT-SPA section: warp tasks pack consecutive checks with at most 32 edges in all
  std::vector<uint16_t> tasks;
  for (int r = 0; r < n_rows;) {
    tasks.push_back((uint16_t)r);
    int edges = 0;
    while (r < n_rows && edges + (row_ptr[r + 1] - row_ptr[r]) <= 32) edges += row_ptr[r + 1] - row_ptr[r], ++r;
    if (edges == 0) ++r;   // a check of degree > 32: its own task (such codes are rejected for q <= 64)
  }
  tasks.push_back((uint16_t)n_rows);
  const int pbits = [&] { int b = 0; while ((1 << b) < q) ++b; return b; }();
  off.edge_row = take(2 * (size_t)nnz);
  off.task_c0 = take(2 * tasks.size());
  off.at_log = take((size_t)(q - 1) * pbits);
  off.fft_bytes = (int)o;
  std::vector<unsigned char> blob(o, 0);
  {
    uint16_t* er = reinterpret_cast<uint16_t*>(&blob[off.edge_row]);
    for (int r = 0; r < n_rows; ++r)
      for (int e = row_ptr[r]; e < row_ptr[r + 1]; ++e) er[e] = (uint16_t)r;
    memcpy(&blob[off.task_c0], tasks.data(), 2 * tasks.size());
    // at_log[lc][i] = M_c^T e_i for c = x^lc: bit k is bit i of c x^k
    uint8_t* at = &blob[off.at_log];
    for (int lc = 0; lc < q - 1; ++lc)
      for (int i = 0; i < pbits; ++i) {
        int a = 0;
        for (int k = 0; k < pbits; ++k) a |= ((exp2[lc + k] >> i) & 1) << k;
        at[lc * pbits + i] = (uint8_t)a;
      }
  }
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
  c->dreg = dmax;                      // regular check degree, or 0 when the rows differ
  for (int r = 0; r < n_rows; ++r)
    if (row_ptr[r + 1] - row_ptr[r] != dmax) c->dreg = 0;
  c->ntasks = (int)tasks.size() - 1;
  c->poly = prim_poly;
  c->off = off;
  if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return NBLDPC_ERR_CUDA; }
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&c->blob_dev), o);
  if (e != cudaSuccess) { delete c; return e == cudaErrorMemoryAllocation ? NBLDPC_ERR_NOMEM : NBLDPC_ERR_CUDA; }
  e = cudaMemcpy(c->blob_dev, blob.data(), o, cudaMemcpyHostToDevice);
  int st = cuda_status(e);
  if (st == NBLDPC_OK) {
    // the resident-message form (384-thread blocks of 1, 2 or 4 frames) must fit shared
    // memory; otherwise the same layout with the messages in the workspace
    const int v = default_variant(q), fpb = default_fpb(c);
    st = v >= 2 ? configure(c, v, (v & 2) && fpb > 4 && !warp4_code(c) ? 4 : fpb) : NBLDPC_ERR_UNSUPPORTED;
    if (st == NBLDPC_ERR_UNSUPPORTED) st = configure(c, v & 1, fpb);
  }
  if (st == NBLDPC_OK) {
    c->fft_status = fft_configure(c);
    if (c->fft_status == NBLDPC_ERR_CUDA) st = NBLDPC_ERR_CUDA;
  }
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

int nbldpc_code_get_tuning(const nbldpc_code* c, int* variant, int* frames_per_block) {
  if (!c) return NBLDPC_ERR_ARG;
  if (variant) *variant = c->variant;
  if (frames_per_block) *frames_per_block = c->plan.fpb;
  return NBLDPC_OK;
}

int nbldpc_code_set_tuning(nbldpc_code* c, int variant, int frames_per_block) {
  if (!c || variant < 0 || variant > 7 || frames_per_block < 1 || frames_per_block > 8 ||
      (frames_per_block & (frames_per_block - 1)))
    return NBLDPC_ERR_ARG;
  const int st = check_device(c);
  if (st != NBLDPC_OK) return st;
  return configure(c, variant, frames_per_block);
}

int nbldpc_code_set_message_bits(nbldpc_code* c, int bits) {
  if (!c || (bits != 8 && bits != 16)) return NBLDPC_ERR_ARG;
  if (bits == 16 && c->cnp_schedule == NBLDPC_CNP_TABLE1) return NBLDPC_ERR_UNSUPPORTED;
  if (check_device(c) != NBLDPC_OK) return check_device(c);
  const int old = c->mb;
  c->mb = bits / 8;
  // resident messages serve 8-bit codes only: a 16-bit code keeps the layout in the workspace form
  const int v = c->mb == 1 ? c->variant : c->variant & 1;
  const int st = configure(c, v, v == c->variant ? c->plan.fpb : 1);
  if (st != NBLDPC_OK) c->mb = old;
  return st;
}

int nbldpc_code_get_message_bits(const nbldpc_code* c, int* bits) {
  if (!c || !bits) return NBLDPC_ERR_ARG;
  *bits = 8 * c->mb;
  return NBLDPC_OK;
}

int nbldpc_code_set_cnp_schedule(nbldpc_code* c, int schedule) {
  if (!c || (schedule != NBLDPC_CNP_MINIMAL && schedule != NBLDPC_CNP_TABLE1)) return NBLDPC_ERR_ARG;
  if (schedule == NBLDPC_CNP_TABLE1 && c->mb != 1) return NBLDPC_ERR_UNSUPPORTED;
  if (check_device(c) != NBLDPC_OK) return check_device(c);
  const int old = c->cnp_schedule;
  c->cnp_schedule = schedule;
  // the schedule is a separate kernel; resident messages serve the minimal schedule only
  const int v = schedule == NBLDPC_CNP_MINIMAL ? c->variant : c->variant & 1;
  const int st = configure(c, v, v == c->variant ? c->plan.fpb : 1);
  if (st != NBLDPC_OK) c->cnp_schedule = old;
  return st;
}

int nbldpc_code_get_cnp_schedule(const nbldpc_code* c, int* schedule) {
  if (!c || !schedule) return NBLDPC_ERR_ARG;
  *schedule = c->cnp_schedule;
  return NBLDPC_OK;
}

int nbldpc_code_set_work_counter(nbldpc_code* c, unsigned long long* counter_dev) {
  if (!c || (counter_dev && !aligned(counter_dev, 8))) return NBLDPC_ERR_ARG;
  c->work_counter = counter_dev;
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
  if (!valid_outputs(gamma_dev, out_sym_dev, out_iters_dev, out_ok_dev) || !workspace_dev) return NBLDPC_ERR_ARG;
  if (!aligned(workspace_dev, 16)) return NBLDPC_ERR_ARG;
  if (workspace_bytes < decode_ws_bytes(c, frames)) return NBLDPC_ERR_ARG;
  int st = check_device(c);
  if (st != NBLDPC_OK) return st;
  st = cuda_status(cudaGetLastError());
  if (st != NBLDPC_OK) return st;
  return launch(c, gamma_dev, frames, max_iters, early_stop, out_sym_dev, out_iters_dev, out_ok_dev,
                workspace_dev, reinterpret_cast<cudaStream_t>(cuda_stream));
}

// ---- mixed-code batches -----------------------------------------------------
static int batch_plan(const nbldpc_job* jobs, int n_jobs, Plan* pl, int* total) {
  if (!jobs || n_jobs < 1 || n_jobs > NBLDPC_MAX_BATCH_JOBS) return NBLDPC_ERR_ARG;
  CodeNeeds need[NBLDPC_MAX_BATCH_JOBS];
  int fpb = 8;
  long long t = 0;
  for (int i = 0; i < n_jobs; ++i) {
    const nbldpc_code* c = jobs[i].code;
    if (!c || jobs[i].frames < 0 || jobs[i].max_iters < 0) return NBLDPC_ERR_ARG;
    const int st = check_device(c);
    if (st != NBLDPC_OK) return st;
    if (kmode(c) != 1) return NBLDPC_ERR_UNSUPPORTED;   // mixed-code launches: 8-bit messages, minimal schedule
    need[i] = needs_of(c, c->variant & 1, 1);
    if (c->plan.fpb < fpb) fpb = c->plan.fpb;
    t += jobs[i].frames;
  }
  if (t > 0x7FFFFFFF) return NBLDPC_ERR_ARG;
  *total = (int)t;
  return make_plan(0, -1, 1, fpb, need, n_jobs, pl);
}

int nbldpc_decode_batch_workspace_size(const nbldpc_job* jobs, int n_jobs, size_t* bytes) {
  if (!bytes) return NBLDPC_ERR_ARG;
  Plan pl{};
  int total = 0;
  const int st = batch_plan(jobs, n_jobs, &pl, &total);
  if (st != NBLDPC_OK) return st;
  *bytes = ws_bytes(pl, total);
  return NBLDPC_OK;
}

int nbldpc_decode_batch(const nbldpc_job* jobs, int n_jobs, void* workspace_dev, size_t workspace_bytes,
                        void* cuda_stream) {
  Plan pl{};
  int total = 0;
  int st = batch_plan(jobs, n_jobs, &pl, &total);
  if (st != NBLDPC_OK) return st;
  if (!workspace_dev || !aligned(workspace_dev, 16) || workspace_bytes < ws_bytes(pl, total)) return NBLDPC_ERR_ARG;
  nbldpc::LaunchParams lp{};
  int begin = 0;
  for (int i = 0; i < n_jobs; ++i) {
    const nbldpc_job& j = jobs[i];
    if (j.frames > 0 && !valid_outputs(j.gamma_dev, j.out_sym_dev, j.out_iters_dev, j.out_ok_dev))
      return NBLDPC_ERR_ARG;
    lp.jobs[i] = job_desc(j.code, j.gamma_dev, j.frames, j.max_iters, j.early_stop, j.out_sym_dev, j.out_iters_dev,
                          j.out_ok_dev, begin);
    begin += j.frames;
  }
  lp.njobs = n_jobs;
  lp.total_items = total;
  st = cuda_status(cudaGetLastError());
  if (st != NBLDPC_OK) return st;
  return launch_plan(kernel_for(0, -1, 1), pl, lp, grid_for(pl, total), workspace_dev,
                     reinterpret_cast<uint8_t*>(workspace_dev) + 256, reinterpret_cast<cudaStream_t>(cuda_stream));
}

// ---- autotuner ----------------------------------------------------------------
constexpr int kTuneReps = 3;         // timed decodes per candidate (the fastest counts)
static size_t tune_outputs(const nbldpc_code* c, int frames) {
  return round_up((size_t)frames * c->n, 256) + round_up((size_t)frames * 4, 256) + round_up((size_t)frames, 256);
}

int nbldpc_code_autotune_workspace_size(const nbldpc_code* c, int frames, size_t* bytes) {
  if (!c || !bytes || frames < 1) return NBLDPC_ERR_ARG;
  size_t mx = 0;
  for (int v = 0; v < 8; ++v)
    for (int fpb = 1; fpb <= 8; fpb *= 2) {
      Plan pl{};
      const CodeNeeds need = needs_of(c, v, c->mb);
      if (make_plan(c->q, v, kmode(c), fpb, &need, 1, &pl) != NBLDPC_OK) continue;
      const size_t w = ws_bytes(pl, frames);
      if (w > mx) mx = w;
    }
  *bytes = tune_outputs(c, frames) + mx;
  return NBLDPC_OK;
}

int nbldpc_code_autotune(nbldpc_code* c, const uint8_t* gamma_dev, int frames, int max_iters, void* workspace_dev,
                         size_t workspace_bytes, void* cuda_stream, nbldpc_tune_result* results, int max_results,
                         int* n_results) {
  if (!c || !gamma_dev || frames < 1 || max_iters < 1 || !workspace_dev || !aligned(gamma_dev, 16) ||
      !aligned(workspace_dev, 256))
    return NBLDPC_ERR_ARG;
  int st = check_device(c);
  if (st != NBLDPC_OK) return st;
  size_t need = 0;
  st = nbldpc_code_autotune_workspace_size(c, frames, &need);
  if (st != NBLDPC_OK) return st;
  if (workspace_bytes < need) return NBLDPC_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  unsigned char* w = reinterpret_cast<unsigned char*>(workspace_dev);
  uint8_t* sym = w;
  int32_t* its = reinterpret_cast<int32_t*>(w + round_up((size_t)frames * c->n, 256));
  uint8_t* okb = w + round_up((size_t)frames * c->n, 256) + round_up((size_t)frames * 4, 256);
  void* dws = w + tune_outputs(c, frames);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return NBLDPC_ERR_CUDA;
  const int v_old = c->variant, f_old = c->plan.fpb;
  int best_v = v_old, best_f = f_old, count = 0;
  float best = 3.4e38f;
  st = NBLDPC_OK;
  for (int v = 0; v < 8 && st == NBLDPC_OK; ++v)
    for (int fpb = 1; fpb <= 8 && st == NBLDPC_OK; fpb *= 2) {
      if (configure(c, v, fpb) != NBLDPC_OK) continue;
      // one untimed decode, then the fastest of kTuneReps timed decodes with fixed iterations
      // (pairs within 1-2 % of each other would otherwise swap places from run to run)
      st = launch(c, gamma_dev, frames, max_iters, 0, sym, its, okb, dws, s, false);
      if (st != NBLDPC_OK) break;
      float ms = 3.4e38f;
      for (int rep = 0; rep < kTuneReps && st == NBLDPC_OK; ++rep) {
        float t = 0.f;
        if (cudaEventRecord(e0, s) != cudaSuccess) { st = NBLDPC_ERR_CUDA; break; }
        st = launch(c, gamma_dev, frames, max_iters, 0, sym, its, okb, dws, s, false);
        if (st != NBLDPC_OK) break;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
          st = NBLDPC_ERR_CUDA;
          break;
        }
        if (t < ms) ms = t;
      }
      if (st != NBLDPC_OK) break;
      if (results && count < max_results) results[count] = nbldpc_tune_result{v, fpb, ms};
      ++count;
      if (ms < best) { best = ms; best_v = v; best_f = fpb; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const int st2 = configure(c, st == NBLDPC_OK ? best_v : v_old, st == NBLDPC_OK ? best_f : f_old);
  if (n_results) *n_results = count;
  return st != NBLDPC_OK ? st : st2;
}

int nbldpc_decode_host_workspace_size(const nbldpc_code* c, int chunk_frames, size_t* bytes) {
  if (!c || !bytes || chunk_frames <= 0) return NBLDPC_ERR_ARG;
  *bytes = 2 * host_chunk_bytes(c, chunk_frames, (size_t)c->n * c->q, decode_ws_bytes(c, chunk_frames));
  return NBLDPC_OK;
}

int nbldpc_decode_host(const nbldpc_code* cc, const uint8_t* gamma_host, int frames, int max_iters, int early_stop,
                       uint8_t* out_sym_host, int32_t* out_iters_host, uint8_t* out_ok_host, int chunk_frames,
                       void* workspace_dev, size_t workspace_bytes, void* cuda_stream) {
  nbldpc_code* c = const_cast<nbldpc_code*>(cc);
  if (!c || frames < 0 || max_iters < 0 || chunk_frames <= 0) return NBLDPC_ERR_ARG;
  if (frames == 0) return NBLDPC_OK;
  const int st = check_device(c);
  if (st != NBLDPC_OK) return st;
  const size_t per = host_chunk_bytes(c, chunk_frames, (size_t)c->n * c->q, decode_ws_bytes(c, chunk_frames));
  return host_chunks(c, gamma_host, (size_t)c->n * c->q, frames, out_sym_host, out_iters_host, out_ok_host,
                     chunk_frames, workspace_dev, workspace_bytes, per, cuda_stream,
                     [&](const void* in, int nf, uint8_t* sy, int32_t* it, uint8_t* okb, void* ws, cudaStream_t s) {
                       return launch(c, reinterpret_cast<const uint8_t*>(in), nf, max_iters, early_stop, sy, it, okb,
                                     ws, s);
                     });
}

}  // extern "C"
