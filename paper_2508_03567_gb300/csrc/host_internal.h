// Host-side internals shared by the C-ABI translation units: nbldpc.cu (code
// handles, min-max decodes, mixed batches, the autotuner) and fftspa_host.cu
// (FFT-SPA decodes).  Not part of the public interface (include/nbldpc.h).
#pragma once

#include "nbldpc.h"

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>

#include "mma_kernels.cuh"   // CodeBlob

namespace nbldpc_host {

// Launch shape of one kernel for one set of codes.
struct Plan {
  int fpb = 1;          // frame slots per block
  int threads = 256;    // block size
  int slot_smem = 0;    // shared bytes per frame slot
  int smem = 0;         // shared bytes per block
  int per_sm = 0;       // resident blocks per SM
  int grid_max = 0;     // resident blocks on the device
  int blob_cap = 0, n_cap = 0;
  size_t slot_bytes = 0;  // message slot per frame slot in the workspace (0: messages in shared memory)
  int xs_off = 0;         // shared-memory offset of the messages (resident launches)
};

extern std::atomic<uint64_t> g_launches;   // decode-kernel launches (nbldpc_kernel_launch_count)
extern std::mutex g_attr_mu;               // guards the per-device kernel attribute flags

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? NBLDPC_OK : NBLDPC_ERR_CUDA; }

inline size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// persistent grid for `frames` frames: at most the resident blocks of the device
inline int grid_for(const Plan& pl, int frames) {
  const int want = (frames + pl.fpb - 1) / pl.fpb;
  return want < pl.grid_max ? want : pl.grid_max;
}

// workspace: a 256-byte frame counter, then one message slot per frame slot of the grid
inline size_t ws_bytes(const Plan& pl, int frames) {
  return 256 + (size_t)grid_for(pl, frames) * pl.fpb * pl.slot_bytes;
}

}  // namespace nbldpc_host

struct nbldpc_code {
  int q = 0, p = 0, n = 0, m = 0, nnz = 0, dmax = 0, vmax = 0;
  uint32_t poly = 0;
  int device = 0;
  unsigned char* blob_dev = nullptr;
  nbldpc::CodeBlob off{};
  int variant = 0;                     // tuning variant used by every decode of this code
  int dreg = 0;                        // degree of every check when all are equal, else 0
  unsigned long long* work_counter = nullptr;   // device counter of visited convolution pairs (optional)
  int mb = 1;                          // message bytes per symbol (1: 8-bit messages, 2: 16-bit)
  int cnp_schedule = NBLDPC_CNP_MINIMAL;   // check-node convolutions: 3(d-2) or Table 1's 3d-4
  nbldpc_host::Plan plan{};            // single-code launch shape (fpb chosen by default or by the autotuner)
  int fft_status = NBLDPC_ERR_UNSUPPORTED;   // FFT-SPA launch shape below valid when NBLDPC_OK
  int fft_dc = 0, fft_dv = 0;          // FFT-SPA check-node form (dc 0: lane per edge) and column-degree bucket
  int ntasks = 0;                      // FFT-SPA warp tasks (blob section)
  nbldpc_host::Plan fft_plan{};
  std::mutex mu;                       // guards the lazily created copy stream
  cudaStream_t side = nullptr;         // second stream for the host-buffer decodes
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
};

namespace nbldpc_host {

// Every launch on a handle must run on the device the handle was created on:
// its code description lives in that device's memory.  NBLDPC_ERR_ARG when
// another device is current (checked before anything is queued).
inline int check_device(const nbldpc_code* c) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return NBLDPC_ERR_CUDA;
  return dev == c->device ? NBLDPC_OK : NBLDPC_ERR_ARG;
}

// FFT-SPA launch shape of a code (fftspa_host.cu): NBLDPC_OK, NBLDPC_ERR_UNSUPPORTED
// when no FFT-SPA kernel covers the code, or NBLDPC_ERR_CUDA.
int fft_configure(nbldpc_code* c);

// ---- host-buffer decodes (nbldpc_decode_host, nbldpc_fftspa_decode_host) ------
// One chunk's device buffers: input rows, symbols, iterations, ok flags, decoder workspace.
inline size_t host_chunk_bytes(const nbldpc_code* c, int chunk_frames, size_t in_bytes_per_frame, size_t decode_ws) {
  return round_up((size_t)chunk_frames * in_bytes_per_frame, 256) + round_up((size_t)chunk_frames * c->n, 256) +
         round_up((size_t)chunk_frames * 4, 256) + round_up((size_t)chunk_frames, 256) + round_up(decode_ws, 256);
}

// Decode host rows in chunks: chunk i copies its rows in, decodes and copies its
// outputs back on stream i % 2 (the caller's stream or the code's side stream),
// in buffer half i % 2 of the workspace, so one chunk's copies overlap the other's
// decode.  `per` is one half's size; `dec` queues the decode of one chunk.
template <class Dec>
int host_chunks(nbldpc_code* c, const void* in_host, size_t fbytes, int frames, uint8_t* out_sym_host,
                int32_t* out_iters_host, uint8_t* out_ok_host, int chunk_frames, void* workspace_dev,
                size_t workspace_bytes, size_t per, void* cuda_stream, Dec dec) {
  if (!in_host || !out_sym_host || !out_iters_host || !out_ok_host || !workspace_dev) return NBLDPC_ERR_ARG;
  if (!aligned(workspace_dev, 256) || workspace_bytes < 2 * per) return NBLDPC_ERR_ARG;
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
  const size_t g_b = round_up((size_t)chunk_frames * fbytes, 256), s_b = round_up((size_t)chunk_frames * c->n, 256),
               i_b = round_up((size_t)chunk_frames * 4, 256), o_b = round_up((size_t)chunk_frames, 256);
  cudaStream_t streams[2] = {main, c->side};
  // the side stream starts after work already queued on the caller's stream
  if (cudaEventRecord(c->ev[0], main) != cudaSuccess || cudaStreamWaitEvent(c->side, c->ev[0], 0) != cudaSuccess)
    return NBLDPC_ERR_CUDA;
  const unsigned char* src = reinterpret_cast<const unsigned char*>(in_host);
  for (int f0 = 0, i = 0; f0 < frames; f0 += chunk_frames, ++i) {
    const int nf = frames - f0 < chunk_frames ? frames - f0 : chunk_frames;
    unsigned char* base = reinterpret_cast<unsigned char*>(workspace_dev) + (size_t)(i & 1) * per;
    void* g = base;
    uint8_t* sy = base + g_b;
    int32_t* it = reinterpret_cast<int32_t*>(base + g_b + s_b);
    uint8_t* okb = base + g_b + s_b + i_b;
    void* ws = base + g_b + s_b + i_b + o_b;
    cudaStream_t s = streams[i & 1];
    cudaError_t e = cudaMemcpyAsync(g, src + (size_t)f0 * fbytes, (size_t)nf * fbytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return NBLDPC_ERR_CUDA;
    st = dec(g, nf, sy, it, okb, ws, s);
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

}  // namespace nbldpc_host
