// host_pipe.cu -- host-buffer round trip of an integer batch in chunks, the
// transfers of one chunk overlapping the kernels of the others (see
// hygt_host_roundtrip in include/hygt.h).
#include <cuda_runtime.h>

#include <cstdint>
#include <new>

#include "../../include/hygt.h"

namespace {

constexpr int kSlots = 3;

struct Slot {
  int16_t* d_x = nullptr;
  uint16_t* d_set = nullptr;
  int32_t* d_y = nullptr;
  int16_t* d_xr = nullptr;
  void* d_work = nullptr;
  int* d_status = nullptr;
  cudaStream_t stream = nullptr;
};

}  // namespace

struct hygt_host_pipe_s {
  hygt_plan plan = nullptr;
  int device = 0;
  int n = 0;  // values per block
  int64_t chunk = 0;
  size_t work_bytes = 0;
  Slot slot[kSlots];
};

static void free_pipe(hygt_host_pipe p) {
  if (!p) return;
  for (Slot& s : p->slot) {
    if (s.stream) {
      cudaStreamSynchronize(s.stream);
      cudaStreamDestroy(s.stream);
    }
    cudaFree(s.d_x);
    cudaFree(s.d_set);
    cudaFree(s.d_y);
    cudaFree(s.d_xr);
    cudaFree(s.d_work);
    cudaFree(s.d_status);
  }
  delete p;
}

extern "C" {

hygt_status hygt_host_pipe_create(hygt_host_pipe* out, hygt_plan plan, int64_t chunk_blocks) {
  if (!out) return HYGT_ERR_ARG;
  *out = nullptr;
  int log2n = 0, is_float = 0;
  if (!plan || chunk_blocks < 1 || chunk_blocks > ((int64_t)1 << 26)) return HYGT_ERR_ARG;
  hygt_status st = hygt_plan_info(plan, &log2n, nullptr, nullptr, &is_float);
  if (st != HYGT_OK) return st;
  if (is_float) return HYGT_ERR_UNSUPPORTED;
  hygt_host_pipe p = new (std::nothrow) hygt_host_pipe_s();
  if (!p) return HYGT_ERR_OOM;
  p->plan = plan;
  p->n = 1 << log2n;
  p->chunk = chunk_blocks;
  p->work_bytes = hygt_batch_workspace_bytes(plan, chunk_blocks);
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return HYGT_ERR_CUDA;
  }
  const size_t vals = (size_t)chunk_blocks * p->n;
  for (Slot& s : p->slot) {
    if (cudaMalloc(&s.d_x, vals * 2) != cudaSuccess || cudaMalloc(&s.d_set, chunk_blocks * 2) != cudaSuccess ||
        cudaMalloc(&s.d_y, vals * 4) != cudaSuccess || cudaMalloc(&s.d_xr, vals * 2) != cudaSuccess ||
        cudaMalloc(&s.d_work, p->work_bytes) != cudaSuccess ||
        cudaMalloc(&s.d_status, sizeof(int)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      free_pipe(p);
      return HYGT_ERR_OOM;
    }
  }
  *out = p;
  return HYGT_OK;
}

hygt_status hygt_host_roundtrip(hygt_host_pipe p, const int16_t* h_x, const uint16_t* h_set,
                                int32_t* h_y, int16_t* h_xr, int64_t nblocks, int* h_status) {
  if (!p || nblocks < 0) return HYGT_ERR_ARG;
  if (h_status) *h_status = 0;
  if (nblocks == 0) return HYGT_OK;
  if (!h_x || !h_xr) return HYGT_ERR_ARG;  // h_y may be null: coefficients stay on the device
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HYGT_ERR_CUDA;
  if (dev != p->device) return HYGT_ERR_ARG;
  for (Slot& s : p->slot)
    if (cudaMemsetAsync(s.d_status, 0, sizeof(int), s.stream) != cudaSuccess) return HYGT_ERR_CUDA;
  const int64_t n = p->n;
  hygt_status st = HYGT_OK;
  int64_t c = 0;
  for (int64_t off = 0; off < nblocks && st == HYGT_OK; off += p->chunk, ++c) {
    Slot& s = p->slot[c % kSlots];
    const int64_t nb = nblocks - off < p->chunk ? nblocks - off : p->chunk;
    cudaStream_t cs = s.stream;
    hygt_stream hs = reinterpret_cast<hygt_stream>(cs);
    // each slot's stream runs its chunks in order, so a slot is reused only
    // after the copies of its previous chunk have left it
    if (cudaMemcpyAsync(s.d_x, h_x + off * n, (size_t)nb * n * 2, cudaMemcpyHostToDevice, cs) !=
        cudaSuccess) {
      st = HYGT_ERR_CUDA;
      break;
    }
    if (h_set && cudaMemcpyAsync(s.d_set, h_set + off, (size_t)nb * 2, cudaMemcpyHostToDevice,
                                 cs) != cudaSuccess) {
      st = HYGT_ERR_CUDA;
      break;
    }
    st = hygt_batch_build(p->plan, h_set ? s.d_set : nullptr, nb, s.d_work, p->work_bytes, hs);
    if (st == HYGT_OK) st = hygt_forward_batch(p->plan, s.d_work, s.d_x, s.d_y, nb, hs, s.d_status);
    if (st == HYGT_OK)
      st = hygt_inverse_batch(p->plan, s.d_work, s.d_y, s.d_xr, nb, hs, s.d_status);
    if (st != HYGT_OK) break;
    if ((h_y && cudaMemcpyAsync(h_y + off * n, s.d_y, (size_t)nb * n * 4, cudaMemcpyDeviceToHost,
                                cs) != cudaSuccess) ||
        cudaMemcpyAsync(h_xr + off * n, s.d_xr, (size_t)nb * n * 2, cudaMemcpyDeviceToHost, cs) !=
            cudaSuccess)
      st = HYGT_ERR_CUDA;
  }
  int first = 0;
  for (Slot& s : p->slot) {
    if (cudaStreamSynchronize(s.stream) != cudaSuccess) st = HYGT_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, s.d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = HYGT_ERR_CUDA;
    if (!first) first = v;
  }
  if (h_status) *h_status = first;
  return st;
}

void hygt_host_pipe_destroy(hygt_host_pipe p) { free_pipe(p); }

}  // extern "C"
