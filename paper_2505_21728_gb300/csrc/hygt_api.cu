// hygt_api.cu -- C ABI of libhygt.so: plan builder (host) and launch entry
// points.  See include/hygt.h for the contract of every call.
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/hygt.h"
#include "hygt_batch.cuh"
#include "hygt_dense.cuh"
#include "hygt_f32b.cuh"
#include "hygt_f32u.cuh"
#include "hygt_fit.cuh"
#include "hygt_secondary.cuh"
#include "hygt_grad.cuh"
#include "hygt_mixed.cuh"
#include "hygt_batch_il.cuh"
#include "hygt_batch_dyn.cuh"
#include "hygt_launch.cuh"

struct hygt_plan_s {
  int log2n = 0, rounds = 0, num_sets = 0;
  int angle_bits = 0, frac_bits = 0;
  int is_float = 0;  // 1: free FP32 angles only (no integer tables)
  int device = 0;
  void* d_tab_int = nullptr;  // uint32 (c | s << 16) per pair
  size_t tab_int_bytes = 0;   // padded to 16
  void* d_tab_f32 = nullptr;  // float2 (cos, sin) per pair
  size_t tab_f32_bytes = 0;
  uint8_t* d_perm = nullptr;  // uint8 [S][R][N]
  size_t perm_bytes = 0;
  unsigned perm_mask = 0;
  int* d_ktab = nullptr;      // batch path: per-set tables [S][ktab_words]
  int ktab_words = 0;         // words per set, padded to a multiple of 4
  int* d_ktabs[hygt::kBatchLayouts] = {};  // the same per register layout ([0] = d_ktab)
  int ktabs_words[hygt::kBatchLayouts] = {};
  hygt::BatchTune tune[2];    // batch path launch tuning: forward, inverse
  int tail[2] = {0, 0};       // dynamic tail of the batch path, 64ths of the tasks
};

namespace hygt {

DeviceInfo device_info(int device) {
  static std::mutex mu;
  static std::vector<DeviceInfo> cache;
  std::lock_guard<std::mutex> lock(mu);
  if ((int)cache.size() <= device) cache.resize(device + 1);
  DeviceInfo& d = cache[device];
  if (d.sms == 0) {
    cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (d.sms <= 0) d.sms = 1;
  }
  return d;
}

}  // namespace hygt

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
// Largest batch of the bucketed path: slots are int32 and each of the
// num_sets + 2 buckets may add 31 padding slots.
constexpr int64_t kBatchMaxBlocks = (int64_t)1 << 30;

size_t pad16(size_t b) { return (b + 15) & ~(size_t)15; }

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

void free_plan(hygt_plan p) {
  if (!p) return;
  if (p->d_tab_int) cudaFree(p->d_tab_int);
  if (p->d_tab_f32) cudaFree(p->d_tab_f32);
  if (p->d_perm) cudaFree(p->d_perm);
  if (p->d_ktab) cudaFree(p->d_ktab);
  for (int l = 1; l < hygt::kBatchLayouts; ++l)
    if (p->d_ktabs[l]) cudaFree(p->d_ktabs[l]);
  delete p;
}

hygt_status upload(void** dst, const void* src, size_t bytes, size_t padded) {
  if (cudaMalloc(dst, padded) != cudaSuccess) {
    *dst = nullptr;
    cudaGetLastError();
    return HYGT_ERR_OOM;
  }
  if (padded > bytes && cudaMemset(*dst, 0, padded) != cudaSuccess) return HYGT_ERR_CUDA;
  if (cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return HYGT_ERR_CUDA;
  return HYGT_OK;
}

bool shape_ok(int log2n, int rounds, int num_sets) {
  return log2n >= 1 && log2n <= HYGT_MAX_LOG2N && rounds >= 1 && rounds <= HYGT_MAX_ROUNDS &&
         num_sets >= 1 && num_sets <= 65535;
}

// Validates the permutation slots (each a permutation of 0..N-1) and
// narrows them to uint8; identity slots are left out of *mask so the
// kernels skip them.  Host only: no CUDA call.
hygt_status check_perms(int log2n, int rounds, int num_sets, const uint16_t* h_perms,
                        std::vector<uint8_t>* out, unsigned* mask) {
  *mask = 0;
  if (!h_perms) return HYGT_OK;
  const int N = 1 << log2n;
  const size_t count = (size_t)num_sets * rounds * N;
  out->assign(count, 0);
  std::vector<int> seen(N);
  for (int s = 0; s < num_sets; ++s) {
    for (int r = 0; r < rounds; ++r) {
      const uint16_t* src = h_perms + ((size_t)s * rounds + r) * N;
      std::fill(seen.begin(), seen.end(), 0);
      bool identity = true;
      for (int i = 0; i < N; ++i) {
        if (src[i] >= N || seen[src[i]]) return HYGT_ERR_ARG;
        seen[src[i]] = 1;
        if (src[i] != i) identity = false;
        (*out)[((size_t)s * rounds + r) * N + i] = (uint8_t)src[i];
      }
      if (!identity) *mask |= 1u << r;
    }
  }
  return HYGT_OK;
}

hygt_status upload_perms(hygt_plan p, const std::vector<uint8_t>& perm, unsigned mask) {
  p->perm_mask = mask;
  if (!mask) return HYGT_OK;
  p->perm_bytes = pad16(perm.size());
  return upload(reinterpret_cast<void**>(&p->d_perm), perm.data(), perm.size(), p->perm_bytes);
}

// Region layout of one permutation slot of the batch kernels (see
// hygt::perm_region_words): word[x] = L q(x) + c(x) for element x, with the
// L-colouring c found as L successive perfect matchings of the bipartite
// multigraph joining each element's natural group (x mod E) to its source
// group (the register index i of the position it is gathered to).  Removing
// a perfect matching from an L-regular bipartite multigraph leaves an
// (L-1)-regular one, so every step succeeds.  Host only.
std::vector<int> perm_region_layout(int N, int E, const uint8_t* perm) {
  const int L = N / E;
  std::vector<int> word(N);
  if (L == 1) {
    for (int x = 0; x < N; ++x) word[x] = x;
    return word;
  }
  std::vector<int> pos(N);  // pos[x]: position gathering element x
  for (int e = 0; e < N; ++e) pos[perm[e]] = e;
  std::vector<int> color(N, -1), match(E);
  std::vector<char> seen(E);
  // augmenting path from natural group w over uncoloured elements (Kuhn)
  std::function<bool(int)> augment = [&](int w) -> bool {
    for (int l = 0; l < L; ++l) {
      const int x = l * E + w;
      if (color[x] >= 0) continue;
      const int r = pos[x] % E;
      if (seen[r]) continue;
      seen[r] = 1;
      if (match[r] < 0 || augment(match[r] % E)) {
        match[r] = x;
        return true;
      }
    }
    return false;
  };
  for (int c = 0; c < L; ++c) {
    std::fill(match.begin(), match.end(), -1);
    for (int w = 0; w < E; ++w) {
      std::fill(seen.begin(), seen.end(), 0);
      if (!augment(w)) return {};
    }
    for (int r = 0; r < E; ++r) color[match[r]] = c;
  }
  std::vector<int> count(L, 0);
  for (int x = 0; x < N; ++x) word[x] = L * count[color[x]]++ + color[x];
  return word;
}

// Per-set tables of the batch kernels (layout: hygt::SetTableShape) for
// 2^log2e values per lane.  Register passes store (c, s - c, -(c + s)) per
// pair in per-lane segments; lane passes store (c, s) for the m side and
// (c, -s) for the n side of each pair; then the permutation gather sources
// as byte offsets in a block's permutation region, per lane.  all_reg (the
// transposed layout, E = N / E values per lane): passes p >= log2e are
// register passes of the transposed block, and the permutation slot reads
// the transposed block and writes the natural one.
bool build_ktab(int log2n, int log2e, int rounds, int num_sets, const uint8_t* q,
                const std::vector<int>& ct, const std::vector<int>& st,
                const std::vector<uint8_t>& perm, unsigned mask, std::vector<int>* out,
                int* words, bool all_reg = false) {
  const int N = 1 << log2n;
  hygt::SetTableShape sh{log2n, log2e, rounds, mask ? 1 : 0};
  sh.all_reg = all_reg;
  if (all_reg && 2 * log2e != log2n) return false;
  const int E = sh.e();
  const int w = (sh.set_words() + 3) & ~3;
  *words = w;
  out->assign((size_t)num_sets * w, 0);
  for (int s = 0; s < num_sets; ++s) {
    int* t = out->data() + (size_t)s * w;
    for (int r = 0; r < rounds; ++r) {
      for (int p = 0; p < log2n; ++p) {
        int* row = t + r * sh.round_words() + sh.pass_offset(p);
        const uint8_t* qa = q + (((size_t)s * rounds + r) * log2n + p) * (N / 2);
        for (int j = 0; j < N / 2; ++j) {
          const int c = ct[qa[j]], sn = st[qa[j]];
          if (p < sh.log2e) {  // lane j / (E/2), pair j mod (E/2) of its segment
            int* e3 = row + (j / (E / 2)) * sh.seg() + 3 * (j % (E / 2));
            e3[0] = c;
            e3[1] = sn - c;
            e3[2] = -(c + sn);
          } else if (all_reg) {
            // transposed block: lane l holds elements (i << log2e) + l; the
            // pair's m side m = (im << log2e) + l with im the register index
            // of its slot jl (the kernel's register-pass order for bit p - log2e)
            const int m = ((((j >> p) << (p + 1)) | (j & ((1 << p) - 1))));
            const int l = m & (E - 1), im = m >> log2e, pb = p - log2e;
            const int jl = ((im >> (pb + 1)) << pb) | (im & ((1 << pb) - 1));
            int* e3 = row + l * sh.seg() + 3 * jl;
            e3[0] = c;
            e3[1] = sn - c;
            e3[2] = -(c + sn);
          } else {
            int* m = row + sh.lane_word(j, 0);
            int* n = row + sh.lane_word(j, 1);
            m[0] = c;
            m[1] = sn;
            n[0] = c;
            n[1] = -sn;
          }
        }
      }
      if (mask) {
        std::vector<uint8_t> ident(N);
        for (int i = 0; i < N; ++i) ident[i] = (uint8_t)i;
        const uint8_t* pr = perm.empty() ? ident.data() : perm.data() + ((size_t)s * rounds + r) * N;
        if (!all_reg) {
          const std::vector<int> word = perm_region_layout(N, E, pr);
          if (word.empty()) return false;
          for (int l = 0; l < N / E; ++l) {
            uint8_t* b = reinterpret_cast<uint8_t*>(t + sh.perm_offset(r) + l * sh.perm_seg());
            for (int i = 0; i < E; ++i) {
              b[i] = (uint8_t)word[l * E + i];
              b[E + i] = (uint8_t)word[pr[l * E + i]];
            }
          }
        } else {
          // The slot is written from the transposed block (lane l, register
          // i' holds element i' E + l) and read as the natural one.  Relabel
          // element x = a E + b as tr(x) = b E + a: the elements one register
          // index of the transposed block writes are then one natural group,
          // and the colouring of perm_region_layout keeps both the writes and
          // the gathered reads on distinct banks; the word of x is that of tr(x).
          auto tr = [&](int x) { return ((x & (E - 1)) << log2e) | (x >> log2e); };
          std::vector<uint8_t> pt(N);
          for (int e = 0; e < N; ++e) pt[e] = (uint8_t)tr(pr[e]);
          const std::vector<int> word = perm_region_layout(N, E, pt.data());
          if (word.empty()) return false;
          for (int l = 0; l < N / E; ++l) {
            uint8_t* b = reinterpret_cast<uint8_t*>(t + sh.perm_offset(r) + l * sh.perm_seg());
            for (int i = 0; i < E; ++i) {
              b[i] = (uint8_t)word[tr((i << log2e) + l)];
              b[E + i] = (uint8_t)word[tr(pr[l * E + i])];
            }
          }
        }
      }
    }
  }
  return true;
}

hygt_status check_io(hygt_plan plan, const void* in, const void* out, int64_t nblocks) {
  if (!plan || nblocks < 0) return HYGT_ERR_ARG;
  if (nblocks == 0) return HYGT_OK;
  if (!in || !out || !aligned16(in) || !aligned16(out)) return HYGT_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HYGT_ERR_CUDA;
  if (dev != plan->device) return HYGT_ERR_ARG;
  return HYGT_OK;
}

hygt::Params base_params(hygt_plan plan, const void* in, void* out, const uint16_t* d_set,
                         int64_t nblocks, int* d_status, bool fp) {
  hygt::Params p{};
  p.in = in;
  p.out = out;
  p.set = d_set;
  p.nblocks = nblocks;
  p.tab = fp ? plan->d_tab_f32 : plan->d_tab_int;
  const size_t tb = fp ? plan->tab_f32_bytes : plan->tab_int_bytes;
  p.tab_bytes = tb > (size_t)INT32_MAX ? 0 : (int)tb;  // 0: never staged
  p.perm = plan->d_perm;
  p.perm_bytes = (int)plan->perm_bytes;
  p.perm_mask = plan->perm_mask;
  p.rounds = plan->rounds;
  p.num_sets = plan->num_sets;
  p.frac_bits = plan->frac_bits;
  p.status = d_status;
  return p;
}

hygt_status to_status(cudaError_t e) {
  if (e == cudaSuccess) return HYGT_OK;
  if (e == cudaErrorMemoryAllocation) return HYGT_ERR_OOM;
  return HYGT_ERR_CUDA;
}

}  // namespace

extern "C" {

hygt_status hygt_create(hygt_plan* out, int log2n, int rounds, int num_sets,
                        const uint8_t* h_angle_idx, const uint16_t* h_perms, int angle_bits,
                        int frac_bits) {
  if (!out) return HYGT_ERR_ARG;
  *out = nullptr;
  if (!shape_ok(log2n, rounds, num_sets) || !h_angle_idx) return HYGT_ERR_ARG;
  if (angle_bits < 1 || angle_bits > 8 || frac_bits < 1 || frac_bits > 10) return HYGT_ERR_ARG;
  const int N = 1 << log2n;
  const size_t pairs = (size_t)num_sets * rounds * log2n * (N / 2);
  const int nq = 1 << angle_bits;
  for (size_t i = 0; i < pairs; ++i)
    if (h_angle_idx[i] >= nq) return HYGT_ERR_ARG;
  std::vector<uint8_t> perm;
  unsigned mask = 0;
  if (check_perms(log2n, rounds, num_sets, h_perms, &perm, &mask) != HYGT_OK) return HYGT_ERR_ARG;

  // Multiplier table of the on-the-fly conversion: c, s = round(2^f cos/sin).
  std::vector<int> ct(nq), st(nq);
  std::vector<float> cf(nq), sf(nq);
  const double scale = std::ldexp(1.0, frac_bits);
  for (int q = 0; q < nq; ++q) {
    const double th = kTwoPi * (double)q / (double)nq;
    ct[q] = (int)std::lround(scale * std::cos(th));
    st[q] = (int)std::lround(scale * std::sin(th));
    cf[q] = (float)std::cos(th);
    sf[q] = (float)std::sin(th);
  }
  std::vector<uint32_t> ti(pairs);
  std::vector<float> tf(2 * pairs);
  for (size_t i = 0; i < pairs; ++i) {
    const int q = h_angle_idx[i];
    ti[i] = ((uint32_t)ct[q] & 0xffffu) | ((uint32_t)st[q] << 16);
    tf[2 * i] = cf[q];
    tf[2 * i + 1] = sf[q];
  }

  hygt_plan p = new (std::nothrow) hygt_plan_s();
  if (!p) return HYGT_ERR_OOM;
  p->log2n = log2n;
  p->rounds = rounds;
  p->num_sets = num_sets;
  p->angle_bits = angle_bits;
  p->frac_bits = frac_bits;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return HYGT_ERR_CUDA;
  }
  hygt_status s = HYGT_OK;
  p->tab_int_bytes = pad16(pairs * 4);
  s = upload(&p->d_tab_int, ti.data(), pairs * 4, p->tab_int_bytes);
  if (s == HYGT_OK) {
    p->tab_f32_bytes = pad16(pairs * 8);
    s = upload(&p->d_tab_f32, tf.data(), pairs * 8, p->tab_f32_bytes);
  }
  if (s == HYGT_OK) s = upload_perms(p, perm, mask);
  if (s == HYGT_OK) {
    std::vector<int> kt;
    if (!build_ktab(log2n, hygt::batch_log2e(log2n), rounds, num_sets, h_angle_idx, ct, st, perm,
                    mask, &kt, &p->ktab_words)) {
      free_plan(p);
      return HYGT_ERR_ARG;
    }
    s = upload(reinterpret_cast<void**>(&p->d_ktab), kt.data(), kt.size() * 4, kt.size() * 4);
    p->d_ktabs[0] = p->d_ktab;
    p->ktabs_words[0] = p->ktab_words;
    for (int l = 1; l < hygt::kBatchLayouts && s == HYGT_OK; ++l) {
      if (!hygt::batch_layout_ok(log2n, l)) continue;
      if (!build_ktab(log2n, hygt::batch_log2e(log2n, l), rounds, num_sets, h_angle_idx, ct, st,
                      perm, mask, &kt, &p->ktabs_words[l], hygt::batch_layout_all_reg(l))) {
        free_plan(p);
        return HYGT_ERR_ARG;
      }
      s = upload(reinterpret_cast<void**>(&p->d_ktabs[l]), kt.data(), kt.size() * 4,
                 kt.size() * 4);
    }
  }
  if (s != HYGT_OK) {
    free_plan(p);
    return s;
  }
  *out = p;
  return HYGT_OK;
}

hygt_status hygt_create_float(hygt_plan* out, int log2n, int rounds, int num_sets,
                              const float* h_theta, const uint16_t* h_perms) {
  if (!out) return HYGT_ERR_ARG;
  *out = nullptr;
  if (!shape_ok(log2n, rounds, num_sets) || !h_theta) return HYGT_ERR_ARG;
  const int N = 1 << log2n;
  const size_t pairs = (size_t)num_sets * rounds * log2n * (N / 2);
  std::vector<float> tf(2 * pairs);
  for (size_t i = 0; i < pairs; ++i) {
    const double th = (double)h_theta[i];
    if (!std::isfinite(th)) return HYGT_ERR_ARG;
    tf[2 * i] = (float)std::cos(th);
    tf[2 * i + 1] = (float)std::sin(th);
  }
  std::vector<uint8_t> perm;
  unsigned mask = 0;
  if (check_perms(log2n, rounds, num_sets, h_perms, &perm, &mask) != HYGT_OK) return HYGT_ERR_ARG;
  hygt_plan p = new (std::nothrow) hygt_plan_s();
  if (!p) return HYGT_ERR_OOM;
  p->log2n = log2n;
  p->rounds = rounds;
  p->num_sets = num_sets;
  p->is_float = 1;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return HYGT_ERR_CUDA;
  }
  p->tab_f32_bytes = pad16(pairs * 8);
  hygt_status s = upload(&p->d_tab_f32, tf.data(), pairs * 8, p->tab_f32_bytes);
  if (s == HYGT_OK) s = upload_perms(p, perm, mask);
  if (s != HYGT_OK) {
    free_plan(p);
    return s;
  }
  *out = p;
  return HYGT_OK;
}

void hygt_destroy(hygt_plan plan) { free_plan(plan); }

hygt_status hygt_forward(hygt_plan plan, const int16_t* d_x, int32_t* d_y, const uint16_t* d_set,
                         int64_t nblocks, hygt_stream stream, int* d_status) {
  hygt_status s = check_io(plan, d_x, d_y, nblocks);
  if (s != HYGT_OK || nblocks == 0) return s;
  if (plan->is_float) return HYGT_ERR_UNSUPPORTED;
  hygt::Params p = base_params(plan, d_x, d_y, d_set, nblocks, d_status, false);
  return to_status(hygt::launch_int_fwd(plan->log2n, p, (cudaStream_t)stream));
}

hygt_status hygt_inverse(hygt_plan plan, const int32_t* d_y, int16_t* d_x, const uint16_t* d_set,
                         int64_t nblocks, hygt_stream stream, int* d_status) {
  hygt_status s = check_io(plan, d_y, d_x, nblocks);
  if (s != HYGT_OK || nblocks == 0) return s;
  if (plan->is_float) return HYGT_ERR_UNSUPPORTED;
  hygt::Params p = base_params(plan, d_y, d_x, d_set, nblocks, d_status, false);
  return to_status(hygt::launch_int_inv(plan->log2n, p, (cudaStream_t)stream));
}

// FP32 transform.  Without set indices every block uses set 0: the one-set
// kernels (four blocks per lane group, the set's table in shared memory);
// with set indices, the direct kernels.
static hygt_status f32_call(hygt_plan plan, const float* in, float* out, const uint16_t* d_set,
                            int64_t nblocks, hygt_stream stream, int* d_status, bool inverse) {
  hygt_status s = check_io(plan, in, out, nblocks);
  if (s != HYGT_OK || nblocks == 0) return s;
  if (!d_set) {
    hygt::F32uParams u{};
    u.in = in;
    u.out = out;
    u.nblocks = nblocks;
    u.tab = static_cast<const float2*>(plan->d_tab_f32);
    u.perm = plan->d_perm;
    u.perm_mask = plan->perm_mask;
    u.rounds = plan->rounds;
    const cudaError_t e = hygt::launch_f32u(plan->log2n, inverse ? 1 : 0, u, (cudaStream_t)stream);
    if (e != cudaErrorInvalidConfiguration) return to_status(e);
    cudaGetLastError();  // table too large for shared memory: direct kernels
  }
  hygt::Params p = base_params(plan, in, out, d_set, nblocks, d_status, true);
  return to_status(inverse ? hygt::launch_f32_inv(plan->log2n, p, (cudaStream_t)stream)
                           : hygt::launch_f32_fwd(plan->log2n, p, (cudaStream_t)stream));
}

hygt_status hygt_forward_f32(hygt_plan plan, const float* d_x, float* d_y, const uint16_t* d_set,
                             int64_t nblocks, hygt_stream stream, int* d_status) {
  return f32_call(plan, d_x, d_y, d_set, nblocks, stream, d_status, false);
}

hygt_status hygt_inverse_f32(hygt_plan plan, const float* d_y, float* d_x, const uint16_t* d_set,
                             int64_t nblocks, hygt_stream stream, int* d_status) {
  return f32_call(plan, d_y, d_x, d_set, nblocks, stream, d_status, true);
}

size_t hygt_batch_workspace_bytes(hygt_plan plan, int64_t nblocks) {
  if (!plan || nblocks < 0 || nblocks > kBatchMaxBlocks) return 0;
  return hygt::batch_layout(plan->num_sets, nblocks, hygt::batch_group(plan->log2n)).total +
         hygt::kDynCounterBytes;
}

// The schedule of a batch, then the dynamic tail's counters zeroed.
static cudaError_t build_schedule(const uint16_t* d_set, int64_t nblocks, int num_sets,
                                  int group, void* d_work, cudaStream_t stream) {
  cudaError_t e = hygt::batch_build(d_set, nblocks, num_sets, group, d_work, stream);
  if (e != cudaSuccess) return e;
  const size_t total = hygt::batch_layout(num_sets, nblocks, group).total;
  return cudaMemsetAsync(static_cast<char*>(d_work) + total, 0, hygt::kDynCounterBytes, stream);
}

// The dynamic tail's counters of a schedule workspace.
static void* tail_counters(hygt_plan plan, const void* d_work, int64_t nblocks) {
  const size_t total =
      hygt::batch_layout(plan->num_sets, nblocks, hygt::batch_group(plan->log2n)).total;
  return const_cast<char*>(static_cast<const char*>(d_work)) + total;
}

hygt_status hygt_batch_build(hygt_plan plan, const uint16_t* d_set, int64_t nblocks, void* d_work,
                             size_t work_bytes, hygt_stream stream) {
  if (!plan || nblocks < 0 || nblocks > kBatchMaxBlocks || !d_work || !aligned16(d_work))
    return HYGT_ERR_ARG;
  const int group = hygt::batch_group(plan->log2n);
  if (work_bytes < hygt_batch_workspace_bytes(plan, nblocks)) return HYGT_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HYGT_ERR_CUDA;
  if (dev != plan->device) return HYGT_ERR_ARG;
  return to_status(
      build_schedule(d_set, nblocks, plan->num_sets, group, d_work, (cudaStream_t)stream));
}

static hygt::BatchParams make_batch_params(hygt_plan plan, const void* d_work, const void* in,
                                           void* out, int64_t nblocks, int* d_status) {
  const hygt::BatchLayout L =
      hygt::batch_layout(plan->num_sets, nblocks, hygt::batch_group(plan->log2n));
  const char* w = static_cast<const char*>(d_work);
  hygt::BatchParams p{};
  p.in = in;
  p.out = out;
  p.order = reinterpret_cast<const int*>(w + L.order);
  p.starts = reinterpret_cast<const int*>(w + L.starts);
  p.meta = reinterpret_cast<const int*>(w + L.meta);
  p.nblocks = nblocks;
  p.tmax = L.tmax;
  p.ktab = plan->d_ktab;
  p.set_words = plan->ktab_words;
  for (int l = 0; l < hygt::kBatchLayouts; ++l) {
    p.ktabs[l] = plan->d_ktabs[l];
    p.set_words_of[l] = plan->ktabs_words[l];
  }
  p.perm_mask = plan->perm_mask;
  p.perms = plan->perm_mask ? 1 : 0;
  p.rounds = plan->rounds;
  p.num_sets = plan->num_sets;
  p.frac_bits = plan->frac_bits;
  p.status = d_status;
  return p;
}

// A bucketed launch in the plan's tuning: stage 4 is the set-interleaved
// order, a nonzero tail the kernels with a dynamic tail, the others the
// batch kernels' own.
static cudaError_t launch_batch_tuned(bool inverse, int log2n, const hygt::BatchParams& p,
                                      cudaStream_t stream, const hygt::BatchTune& tune,
                                      int tail = 0, void* counters = nullptr) {
  if (tune.stage == 4) return hygt::launch_batch_il(inverse ? 1 : 0, log2n, p, stream, tune);
  if (tail > 0)
    return hygt::launch_batch_dyn(inverse ? 1 : 0, log2n, p, counters, tail, stream, tune);
  return inverse ? hygt::launch_batch_inv(log2n, p, stream, tune)
                 : hygt::launch_batch_fwd(log2n, p, stream, tune);
}

static hygt_status batch_call(hygt_plan plan, const void* d_work, const void* in, void* out,
                              int64_t nblocks, hygt_stream stream, int* d_status, bool inverse) {
  hygt_status s = check_io(plan, in, out, nblocks);
  if (s != HYGT_OK || nblocks == 0) return s;
  if (plan->is_float) return HYGT_ERR_UNSUPPORTED;
  if (!d_work || !aligned16(d_work) || nblocks > kBatchMaxBlocks) return HYGT_ERR_ARG;
  const hygt::BatchParams p = make_batch_params(plan, d_work, in, out, nblocks, d_status);
  cudaError_t e = launch_batch_tuned(inverse, plan->log2n, p, (cudaStream_t)stream,
                                     plan->tune[inverse ? 1 : 0], plan->tail[inverse ? 1 : 0],
                                     tail_counters(plan, d_work, nblocks));
  if (e == cudaErrorInvalidConfiguration) return HYGT_ERR_UNSUPPORTED;
  return to_status(e);
}

hygt_status hygt_forward_batch(hygt_plan plan, const void* d_work, const int16_t* d_x, int32_t* d_y,
                               int64_t nblocks, hygt_stream stream, int* d_status) {
  return batch_call(plan, d_work, d_x, d_y, nblocks, stream, d_status, false);
}

hygt_status hygt_inverse_batch(hygt_plan plan, const void* d_work, const int32_t* d_y, int16_t* d_x,
                               int64_t nblocks, hygt_stream stream, int* d_status) {
  return batch_call(plan, d_work, d_y, d_x, nblocks, stream, d_status, true);
}

static hygt_status batch_f32_call(hygt_plan plan, const void* d_work, const float* in,
                                  float* out, int64_t nblocks, hygt_stream stream, int* d_status,
                                  bool inverse) {
  hygt_status s = check_io(plan, in, out, nblocks);
  if (s != HYGT_OK || nblocks == 0) return s;
  if (plan->log2n < 4) return HYGT_ERR_UNSUPPORTED;
  if (!d_work || !aligned16(d_work) || nblocks > kBatchMaxBlocks) return HYGT_ERR_ARG;
  const int group = hygt::batch_group(plan->log2n);
  const hygt::BatchLayout L = hygt::batch_layout(plan->num_sets, nblocks, group);
  const char* w = static_cast<const char*>(d_work);
  hygt::F32bParams p{};
  p.in = in;
  p.out = out;
  p.nblocks = nblocks;
  p.tab = static_cast<const float2*>(plan->d_tab_f32);
  p.perm = plan->d_perm;
  p.perm_mask = plan->perm_mask;
  p.rounds = plan->rounds;
  p.num_sets = plan->num_sets;
  p.order = reinterpret_cast<const int*>(w + L.order);
  p.starts = reinterpret_cast<const int*>(w + L.starts);
  p.meta = reinterpret_cast<const int*>(w + L.meta);
  p.tmax = L.tmax;
  p.group_sched = group;
  p.status = d_status;
  cudaError_t e = hygt::launch_f32b(plan->log2n, inverse ? 1 : 0, p, (cudaStream_t)stream);
  if (e == cudaErrorInvalidConfiguration) return HYGT_ERR_UNSUPPORTED;
  return to_status(e);
}

hygt_status hygt_forward_batch_f32(hygt_plan plan, const void* d_work, const float* d_x,
                                   float* d_y, int64_t nblocks, hygt_stream stream,
                                   int* d_status) {
  return batch_f32_call(plan, d_work, d_x, d_y, nblocks, stream, d_status, false);
}

hygt_status hygt_inverse_batch_f32(hygt_plan plan, const void* d_work, const float* d_y,
                                   float* d_x, int64_t nblocks, hygt_stream stream,
                                   int* d_status) {
  return batch_f32_call(plan, d_work, d_y, d_x, nblocks, stream, d_status, true);
}

hygt_status hygt_batch_set_tuning(hygt_plan plan, int inverse, int warps_per_cta,
                                  int ctas_per_sm, int stage, int layout) {
  if (!plan || (inverse != 0 && inverse != 1) || warps_per_cta < 0 || ctas_per_sm < 0 ||
      ctas_per_sm > 8 || stage < -1 || stage > 4 || layout < 0 || layout >= hygt::kBatchLayouts)
    return HYGT_ERR_ARG;
  const int max_warps = hygt::batch_threads(plan->log2n, inverse, layout) / 32;
  if (warps_per_cta > max_warps) return HYGT_ERR_ARG;
  if (stage >= 0 && plan->log2n < 4) return HYGT_ERR_UNSUPPORTED;
  if (layout != 0 && (!plan->d_ktabs[layout] || stage == 3)) return HYGT_ERR_UNSUPPORTED;
  if (stage == 4 && !hygt::batch_il_ok(plan->log2n, layout)) return HYGT_ERR_UNSUPPORTED;
  if (plan->tail[inverse] > 0 && !hygt::batch_dyn_ok(plan->log2n, layout, stage))
    return HYGT_ERR_UNSUPPORTED;  // a dynamic tail is set: clear it first
  hygt::BatchTune& t = plan->tune[inverse];
  t.warps = warps_per_cta;
  t.ctas_per_sm = ctas_per_sm;
  t.stage = stage;
  t.layout = layout;
  return HYGT_OK;
}

hygt_status hygt_batch_get_tuning(hygt_plan plan, int inverse, int* warps_per_cta,
                                  int* ctas_per_sm, int* stage, int* layout, int* max_warps) {
  if (!plan || (inverse != 0 && inverse != 1)) return HYGT_ERR_ARG;
  const hygt::BatchTune& t = plan->tune[inverse];
  if (warps_per_cta) *warps_per_cta = t.warps;
  if (ctas_per_sm) *ctas_per_sm = t.ctas_per_sm;
  if (stage) *stage = t.stage;
  if (layout) *layout = t.layout;
  if (max_warps) *max_warps = hygt::batch_threads(plan->log2n, inverse, t.layout) / 32;
  return HYGT_OK;
}

hygt_status hygt_batch_set_tail(hygt_plan plan, int inverse, int tail_64ths) {
  if (!plan || (inverse != 0 && inverse != 1) || tail_64ths < 0 || tail_64ths > 32)
    return HYGT_ERR_ARG;
  const hygt::BatchTune& t = plan->tune[inverse];
  if (tail_64ths > 0 && !hygt::batch_dyn_ok(plan->log2n, t.layout, t.stage))
    return HYGT_ERR_UNSUPPORTED;
  plan->tail[inverse] = tail_64ths;
  return HYGT_OK;
}

hygt_status hygt_batch_get_tail(hygt_plan plan, int inverse, int* tail_64ths) {
  if (!plan || (inverse != 0 && inverse != 1) || !tail_64ths) return HYGT_ERR_ARG;
  *tail_64ths = plan->tail[inverse];
  return HYGT_OK;
}

int hygt_mixed_ctas(void) { return hygt::mixed_grid_ctas(); }

hygt_status hygt_mixed_class_variant(hygt_plan plan, int inverse, int* stage, int* layout) {
  if (!plan) return HYGT_ERR_ARG;
  if (plan->is_float || (plan->log2n != 4 && plan->log2n != 6 && plan->log2n != 8))
    return HYGT_ERR_UNSUPPORTED;
  const hygt::BatchTune& tune = plan->tune[inverse ? 1 : 0];
  const hygt::MixedVariant mv = hygt::mixed_variant(
      plan->log2n, hygt::mixed_variant_of(plan->log2n, tune.stage, tune.layout));
  if (stage) *stage = mv.stage;
  if (layout) *layout = mv.layout;
  return HYGT_OK;
}

// Validates the classes of a mixed launch and fills the kernel parameters.
// How a mixed batch is run (from the classes' `ctas`).
enum MixedMode { kMixedSequential, kMixedConcurrent, kMixedSeparate };

// How one class runs in separate launches: its plan's tuning and dynamic
// tail for the direction, and the tail's counters in its workspace.
struct ClassLaunch {
  hygt::BatchTune tune;
  int tail = 0;
  void* counters = nullptr;
};

static hygt_status mixed_params(const hygt_mixed_class* cls, int nclasses, bool inverse,
                                int* d_status, hygt::MixedParams* mp, MixedMode* mode,
                                ClassLaunch* runs = nullptr) {
  if (!cls || nclasses < 1 || nclasses > hygt::kMaxMixedClasses) return HYGT_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HYGT_ERR_CUDA;
  *mp = hygt::MixedParams{};
  bool explicit_split = true, separate = true;
  int explicit_sum = 0;
  int slot_ctas[hygt::kMaxMixedClasses] = {0, 0, 0};
  bool seen[hygt::kMaxMixedClasses] = {false, false, false};
  for (int c = 0; c < nclasses; ++c) {
    const hygt_mixed_class& k = cls[c];
    hygt_plan plan = k.plan;
    if (!plan || plan->is_float) return plan ? HYGT_ERR_UNSUPPORTED : HYGT_ERR_ARG;
    if (plan->log2n != 4 && plan->log2n != 6 && plan->log2n != 8) return HYGT_ERR_UNSUPPORTED;
    if (plan->device != dev || k.nblocks < 0 || k.nblocks > kBatchMaxBlocks) return HYGT_ERR_ARG;
    const int slot = (plan->log2n - 4) / 2;
    if (seen[slot]) return HYGT_ERR_ARG;  // one class per block size
    seen[slot] = true;
    const void* in = inverse ? (const void*)k.d_y : (const void*)k.d_x;
    void* out = inverse ? (void*)k.d_xr : (void*)k.d_y;
    if (k.nblocks > 0) {
      if (!in || !out || !aligned16(in) || !aligned16(out) || !k.d_work || !aligned16(k.d_work))
        return HYGT_ERR_ARG;
      const int group = hygt::batch_group(plan->log2n);
      if (k.work_bytes < hygt_batch_workspace_bytes(plan, k.nblocks))
        return HYGT_ERR_ARG;
    }
    mp->cls[slot] = make_batch_params(plan, k.d_work, in, out, k.nblocks, d_status);
    mp->present[slot] = k.nblocks > 0 ? 1 : 0;
    const hygt::BatchTune& tune = plan->tune[inverse ? 1 : 0];
    mp->variant[slot] = hygt::mixed_variant_of(plan->log2n, tune.stage, tune.layout);
    if (runs) {
      runs[slot].tune = tune;
      runs[slot].tail = plan->tail[inverse ? 1 : 0];
      runs[slot].counters = k.nblocks > 0 ? tail_counters(plan, k.d_work, k.nblocks) : nullptr;
    }
    slot_ctas[slot] = k.ctas;
    if (k.ctas <= 0) explicit_split = false;
    if (k.ctas != -1) separate = false;
    explicit_sum += k.ctas > 0 ? k.ctas : 0;
  }
  const int grid = hygt::mixed_grid_ctas();
  if (grid < 1) return HYGT_ERR_CUDA;
  mp->cta_begin[0] = 0;
  *mode = separate ? kMixedSeparate
                   : (explicit_split && explicit_sum <= 4 * grid) ? kMixedConcurrent
                                                                   : kMixedSequential;
  if (*mode == kMixedConcurrent) {
    mp->sequential = 0;
    for (int k = 0; k < hygt::kMaxMixedClasses; ++k)
      mp->cta_begin[k + 1] = mp->cta_begin[k] + (mp->present[k] ? slot_ctas[k] : 0);
  } else {
    mp->sequential = 1;  // every CTA takes part in every class, one class after the other
    for (int k = 0; k < hygt::kMaxMixedClasses; ++k) mp->cta_begin[k + 1] = grid;
  }
  return HYGT_OK;
}

// One direction of a mixed batch: the mixed kernel, or (separate mode) the
// batch kernel of each class in turn.
static cudaError_t mixed_launch(const hygt::MixedParams& mp, MixedMode mode, bool inverse,
                                cudaStream_t stream, const ClassLaunch* runs) {
  if (mode != kMixedSeparate) return hygt::launch_mixed(inverse ? 1 : 0, mp, stream);
  for (int k = 0; k < hygt::kMaxMixedClasses; ++k) {
    if (!mp.present[k]) continue;
    const int log2n = hygt::mixed_slot_log2n(k);
    const cudaError_t e = launch_batch_tuned(inverse, log2n, mp.cls[k], stream, runs[k].tune,
                                             runs[k].tail, runs[k].counters);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static hygt_status mixed_call(const hygt_mixed_class* cls, int nclasses, hygt_stream stream,
                              int* d_status, bool inverse) {
  hygt::MixedParams mp;
  MixedMode mode;
  ClassLaunch runs[hygt::kMaxMixedClasses];
  hygt_status s = mixed_params(cls, nclasses, inverse, d_status, &mp, &mode, runs);
  if (s != HYGT_OK) return s;
  const cudaError_t e = mixed_launch(mp, mode, inverse, (cudaStream_t)stream, runs);
  if (e == cudaErrorInvalidConfiguration) return HYGT_ERR_UNSUPPORTED;
  return to_status(e);
}

hygt_status hygt_forward_mixed(const hygt_mixed_class* classes, int nclasses, hygt_stream stream,
                               int* d_status) {
  return mixed_call(classes, nclasses, stream, d_status, false);
}

hygt_status hygt_inverse_mixed(const hygt_mixed_class* classes, int nclasses, hygt_stream stream,
                               int* d_status) {
  return mixed_call(classes, nclasses, stream, d_status, true);
}

struct hygt_graph_s {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

// Streams and events of a capture with one branch per class.
struct GraphBranches {
  cudaStream_t stream[hygt::kMaxMixedClasses] = {};
  cudaEvent_t join[hygt::kMaxMixedClasses] = {};
  cudaEvent_t fork = nullptr;
  ~GraphBranches() {
    for (int k = 0; k < hygt::kMaxMixedClasses; ++k) {
      if (join[k]) cudaEventDestroy(join[k]);
      if (stream[k]) cudaStreamDestroy(stream[k]);
    }
    if (fork) cudaEventDestroy(fork);
  }
};

// The classes' schedules share no data: each is built on a branch of its own
// that forks from and joins `cs`, so the small launches of one schedule (the
// one-CTA scan, the small classes' count and scatter) run beside those of
// the others.  (Branching the transform launches as well was measured slower:
// persistent launches that start on a few SMs at a time finish late.)
static cudaError_t capture_schedules(const hygt_mixed_class* classes, int nclasses,
                                     cudaStream_t cs, GraphBranches& br) {
  cudaError_t e = cudaEventCreateWithFlags(&br.fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(br.fork, cs);
  int nb = 0;
  for (int c = 0; c < nclasses && e == cudaSuccess; ++c) {
    const hygt_mixed_class& k = classes[c];
    if (k.nblocks <= 0) continue;
    e = cudaStreamCreateWithFlags(&br.stream[nb], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&br.join[nb], cudaEventDisableTiming);
    if (e != cudaSuccess) break;
    cudaStream_t s = br.stream[nb];
    e = cudaStreamWaitEvent(s, br.fork, 0);
    if (e == cudaSuccess)
      e = build_schedule(k.d_set, k.nblocks, k.plan->num_sets,
                         hygt::batch_group(k.plan->log2n), k.d_work, s);
    if (e == cudaSuccess) e = cudaEventRecord(br.join[nb], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, br.join[nb], 0);
    ++nb;
  }
  return e;
}

hygt_status hygt_mixed_graph_create(hygt_graph* out, const hygt_mixed_class* classes, int nclasses,
                                    int* d_status) {
  if (!out) return HYGT_ERR_ARG;
  *out = nullptr;
  hygt::MixedParams fwd, inv;
  MixedMode mode;
  ClassLaunch tf[hygt::kMaxMixedClasses], ti[hygt::kMaxMixedClasses];
  hygt_status s = mixed_params(classes, nclasses, false, d_status, &fwd, &mode, tf);
  if (s == HYGT_OK) s = mixed_params(classes, nclasses, true, d_status, &inv, &mode, ti);
  if (s != HYGT_OK) return s;
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return HYGT_ERR_CUDA;
  hygt_graph g = new (std::nothrow) hygt_graph_s();
  if (!g) {
    cudaStreamDestroy(cs);
    return HYGT_ERR_OOM;
  }
  GraphBranches br;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = capture_schedules(classes, nclasses, cs, br);
  if (e == cudaSuccess) e = mixed_launch(fwd, mode, false, cs, tf);
  if (e == cudaSuccess) e = mixed_launch(inv, mode, true, cs, ti);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, graph, 0);
  g->graph = graph;
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    hygt_graph_destroy(g);
    cudaGetLastError();
    return HYGT_ERR_CUDA;
  }
  *out = g;
  return HYGT_OK;
}

hygt_status hygt_graph_launch(hygt_graph graph, hygt_stream stream) {
  if (!graph || !graph->exec) return HYGT_ERR_ARG;
  return to_status(cudaGraphLaunch(graph->exec, (cudaStream_t)stream));
}

void hygt_graph_destroy(hygt_graph graph) {
  if (!graph) return;
  if (graph->exec) cudaGraphExecDestroy(graph->exec);
  if (graph->graph) cudaGraphDestroy(graph->graph);
  delete graph;
}

hygt_status hygt_update_theta(hygt_plan plan, const float* d_theta, hygt_stream stream) {
  if (!plan || !d_theta) return HYGT_ERR_ARG;
  if (!plan->is_float) return HYGT_ERR_UNSUPPORTED;
  const long long n = (long long)plan->num_sets * plan->rounds * plan->log2n * (1 << (plan->log2n - 1));
  hygt::hygt_theta_to_table<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      d_theta, static_cast<float2*>(plan->d_tab_f32), n);
  return to_status(cudaGetLastError());
}

static int plan_angles(hygt_plan plan) {
  return plan->num_sets * plan->rounds * plan->log2n * (1 << (plan->log2n - 1));
}

// Backward workspace: the CTA partials of dL/dtheta, then (used when set
// indices are given) the set-bucketed schedule of the backward's task size.
struct GradWork {
  int threads, grid, cache_tables, group;
  size_t smem, partials, sched_off, total;
};

static GradWork grad_work(hygt_plan plan, int64_t nblocks) {
  GradWork w{};
  hygt::grad_config(plan->log2n, plan->num_sets, plan->rounds, nblocks, &w.threads, &w.grid,
                    &w.smem, &w.cache_tables, &w.group);
  if (w.threads == 0) return w;
  w.partials = (size_t)(w.grid > 0 ? w.grid : 1) * plan_angles(plan) * sizeof(double);
  w.sched_off = hygt::align16(w.partials);
  w.total = w.sched_off + hygt::batch_layout(plan->num_sets, nblocks, w.group).total;
  return w;
}

size_t hygt_backward_workspace_bytes(hygt_plan plan, int64_t nblocks) {
  if (!plan || nblocks < 0 || nblocks > kBatchMaxBlocks) return 0;
  const GradWork w = grad_work(plan, nblocks);
  return w.threads == 0 ? 0 : w.total;
}

// The backward of hygt_backward_f32 (d_gy given) and of hygt_backward_diag_f32
// (d_gy null: dL/dy = w * y, d_gx optional).
static hygt_status backward_common(hygt_plan plan, const float* d_y, const float* d_gy,
                                   const float* d_w, float* d_gx, double* d_gtheta,
                                   const uint16_t* d_set, int64_t nblocks, void* d_work,
                                   size_t work_bytes, hygt_stream stream, int* d_status) {
  const int angles = plan_angles(plan);
  const GradWork w = grad_work(plan, nblocks);
  if (w.threads == 0) return HYGT_ERR_UNSUPPORTED;
  if (!d_work || !aligned16(d_work) || work_bytes < w.total) return HYGT_ERR_ARG;
  if (nblocks == 0) {
    return to_status(cudaMemsetAsync(d_gtheta, 0, (size_t)angles * sizeof(double),
                                     (cudaStream_t)stream));
  }
  hygt::GradLaunch gl{};
  gl.log2n = plan->log2n;
  gl.threads = w.threads;
  gl.grid = w.grid;
  gl.smem = w.smem;
  gl.p.y = d_y;
  gl.p.gy = d_gy;
  gl.p.w = d_w;
  gl.p.gx = d_gx;
  gl.p.nblocks = nblocks;
  gl.p.tab = static_cast<const float2*>(plan->d_tab_f32);
  gl.p.perm = plan->d_perm;
  gl.p.perm_mask = plan->perm_mask;
  gl.p.rounds = plan->rounds;
  gl.p.num_sets = plan->num_sets;
  gl.p.angles = angles;
  gl.p.cache_tables = w.cache_tables;
  gl.p.partials = static_cast<double*>(d_work);
  gl.p.status = d_status;
  if (d_set) {
    // tasks of one set each: bucket the blocks by set
    char* sched = static_cast<char*>(d_work) + w.sched_off;
    const hygt::BatchLayout L = hygt::batch_layout(plan->num_sets, nblocks, w.group);
    cudaError_t e = hygt::batch_build(d_set, nblocks, plan->num_sets, w.group, sched,
                                      (cudaStream_t)stream);
    if (e != cudaSuccess) return to_status(e);
    gl.p.order = reinterpret_cast<const int*>(sched + L.order);
    gl.p.starts = reinterpret_cast<const int*>(sched + L.starts);
    gl.p.meta = reinterpret_cast<const int*>(sched + L.meta);
    gl.p.tmax = L.tmax;
  }
  return to_status(hygt::launch_grad(gl, d_gtheta, (cudaStream_t)stream));
}

hygt_status hygt_backward_f32(hygt_plan plan, const float* d_y, const float* d_gy, float* d_gx,
                              double* d_gtheta, const uint16_t* d_set, int64_t nblocks,
                              void* d_work, size_t work_bytes, hygt_stream stream, int* d_status) {
  if (!plan || nblocks < 0 || nblocks > kBatchMaxBlocks || !d_gtheta) return HYGT_ERR_ARG;
  hygt_status s = check_io(plan, d_y, d_gx, nblocks);
  if (s != HYGT_OK) return s;
  if (nblocks > 0 && (!d_gy || !aligned16(d_gy))) return HYGT_ERR_ARG;
  return backward_common(plan, d_y, d_gy, nullptr, d_gx, d_gtheta, d_set, nblocks, d_work,
                         work_bytes, stream, d_status);
}

hygt_status hygt_backward_diag_f32(hygt_plan plan, const float* d_y, const float* d_w,
                                   float* d_gx, double* d_gtheta, const uint16_t* d_set,
                                   int64_t nblocks, void* d_work, size_t work_bytes,
                                   hygt_stream stream, int* d_status) {
  if (!plan || nblocks < 0 || nblocks > kBatchMaxBlocks || !d_gtheta || !d_w) return HYGT_ERR_ARG;
  if (nblocks > 0 && (!d_y || !aligned16(d_y))) return HYGT_ERR_ARG;
  if (d_gx && (!aligned16(d_gx) || d_gx == (float*)d_y)) return HYGT_ERR_ARG;
  return backward_common(plan, d_y, nullptr, d_w, d_gx, d_gtheta, d_set, nblocks, d_work,
                         work_bytes, stream, d_status);
}

// The secondary-transform pipeline (hygt_secondary.cuh): checks, the
// primary matrix C = round(256 D) of the orthonormal DCT-II, the launch.
static hygt_status secondary_run(int inverse, hygt_plan plan, int log2m, const void* in,
                                 void* out, const uint16_t* d_set, int64_t nblocks,
                                 hygt_stream stream, int* d_status) {
  if (!plan || nblocks < 0 || nblocks > kBatchMaxBlocks) return HYGT_ERR_ARG;
  if (plan->is_float) return HYGT_ERR_UNSUPPORTED;
  if (log2m < 2 || log2m > 5) return HYGT_ERR_ARG;
  // 4x4 blocks take a 4x4 secondary (N = 16), larger blocks an 8x8 one (N = 64)
  if (plan->log2n != (log2m == 2 ? 4 : 6)) return HYGT_ERR_ARG;
  if (nblocks == 0) return HYGT_OK;
  if (!in || !out || !aligned16(in) || !aligned16(out)) return HYGT_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HYGT_ERR_CUDA;
  if (dev != plan->device) return HYGT_ERR_ARG;
  hygt::SecondaryParams p{};
  const int M = 1 << log2m;
  for (int k = 0; k < M; ++k) {
    const double a = k == 0 ? std::sqrt(1.0 / M) : std::sqrt(2.0 / M);
    for (int i = 0; i < M; ++i)
      p.C[k * M + i] = (int16_t)std::lround(256.0 * a * std::cos(kTwoPi * (2.0 * i + 1.0) * k /
                                                                 (4.0 * M)));
  }
  p.in = in;
  p.out = out;
  p.set = d_set;
  p.nblocks = nblocks;
  p.log2m = log2m;
  p.log2n = plan->log2n;
  p.rounds = plan->rounds;
  p.num_sets = plan->num_sets;
  p.frac_bits = plan->frac_bits;
  p.perm_mask = plan->perm_mask;
  p.tab = static_cast<const uint32_t*>(plan->d_tab_int);
  p.perm = plan->d_perm;
  p.group = M * M >= 512 ? 1 : 512 / (M * M);
  p.status = d_status;
  return to_status(hygt::launch_secondary(inverse, p, (cudaStream_t)stream));
}

// The secondary pipeline of 4x4 / 8x8 blocks through the set-bucketed
// kernels with the primary fused (schedule from hygt_batch_build).
static hygt_status secondary_batch_run(int inverse, hygt_plan plan, const void* d_work,
                                       int log2m, const void* in, void* out, int64_t nblocks,
                                       hygt_stream stream, int* d_status) {
  hygt_status s = check_io(plan, in, out, nblocks);
  if (s != HYGT_OK || nblocks == 0) return s;
  if (plan->is_float) return HYGT_ERR_UNSUPPORTED;
  if (log2m != 2 && log2m != 3) return HYGT_ERR_UNSUPPORTED;
  if (plan->log2n != 2 * log2m) return HYGT_ERR_ARG;
  if (!d_work || !aligned16(d_work) || nblocks > kBatchMaxBlocks) return HYGT_ERR_ARG;
  const hygt::BatchParams p = make_batch_params(plan, d_work, in, out, nblocks, d_status);
  cudaError_t e = hygt::launch_batch_primary(plan->log2n, inverse, p, (cudaStream_t)stream,
                                             plan->tune[inverse]);
  if (e == cudaErrorInvalidConfiguration) return HYGT_ERR_UNSUPPORTED;
  return to_status(e);
}

hygt_status hygt_secondary_forward_batch(hygt_plan plan, const void* d_work, int log2m,
                                         const int16_t* d_x, int32_t* d_y, int64_t nblocks,
                                         hygt_stream stream, int* d_status) {
  return secondary_batch_run(0, plan, d_work, log2m, d_x, d_y, nblocks, stream, d_status);
}

hygt_status hygt_secondary_inverse_batch(hygt_plan plan, const void* d_work, int log2m,
                                         const int32_t* d_y, int16_t* d_x, int64_t nblocks,
                                         hygt_stream stream, int* d_status) {
  return secondary_batch_run(1, plan, d_work, log2m, d_y, d_x, nblocks, stream, d_status);
}

hygt_status hygt_secondary_forward(hygt_plan plan, int log2m, const int16_t* d_x, int32_t* d_y,
                                   const uint16_t* d_set, int64_t nblocks, hygt_stream stream,
                                   int* d_status) {
  return secondary_run(0, plan, log2m, d_x, d_y, d_set, nblocks, stream, d_status);
}

hygt_status hygt_secondary_inverse(hygt_plan plan, int log2m, const int32_t* d_y, int16_t* d_x,
                                   const uint16_t* d_set, int64_t nblocks, hygt_stream stream,
                                   int* d_status) {
  return secondary_run(1, plan, log2m, d_y, d_x, d_set, nblocks, stream, d_status);
}

size_t hygt_coding_gain_workspace_bytes(hygt_plan plan, int64_t nblocks) {
  if (!plan || nblocks < 1 || nblocks > kBatchMaxBlocks || plan->log2n < 2) return 0;
  const long long n4 = (long long)nblocks * (1 << plan->log2n) / 4;
  return (size_t)hygt::moments_grid(n4) * (size_t)(1 << plan->log2n) * sizeof(double);
}

hygt_status hygt_coding_gain_f32(hygt_plan plan, const float* d_y, int64_t nblocks, double* d_v,
                                 float* d_w, double* d_J, void* d_work, size_t work_bytes,
                                 hygt_stream stream) {
  if (!plan || nblocks < 1 || nblocks > kBatchMaxBlocks || !d_y || !aligned16(d_y) || !d_v ||
      !d_w || !d_J)
    return HYGT_ERR_ARG;
  if (plan->log2n < 2) return HYGT_ERR_UNSUPPORTED;
  const size_t need = hygt_coding_gain_workspace_bytes(plan, nblocks);
  if (!d_work || !aligned16(d_work) || work_bytes < need) return HYGT_ERR_ARG;
  const int n = 1 << plan->log2n;
  const long long n4 = (long long)nblocks * n / 4;
  const int grid = hygt::moments_grid(n4);
  double* partials = static_cast<double*>(d_work);
  hygt::hygt_moments_kernel<<<grid, hygt::kMomentThreads, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const float4*>(d_y), n4, n, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return to_status(e);
  hygt::hygt_coding_gain_finish<<<1, n, 0, (cudaStream_t)stream>>>(partials, grid, n, nblocks,
                                                                   d_v, d_w, d_J);
  return to_status(cudaGetLastError());
}

hygt_status hygt_adam_step(float* d_theta, const double* d_grad, float* d_m, float* d_v,
                           int64_t n, float lr, float beta1, float beta2, float eps, int step,
                           hygt_stream stream) {
  if (!d_theta || !d_grad || !d_m || !d_v || n < 1 || step < 1 || !(lr > 0.f) ||
      !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return HYGT_ERR_ARG;
  const float corr1 = 1.f - (float)std::pow((double)beta1, (double)step);
  const float corr2 = 1.f - (float)std::pow((double)beta2, (double)step);
  hygt::hygt_adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      d_theta, d_grad, d_m, d_v, n, lr, beta1, beta2, eps, corr1 > 0.f ? corr1 : 1.f,
      corr2 > 0.f ? corr2 : 1.f);
  return to_status(cudaGetLastError());
}

struct dense_klt_s {
  int log2n = 0, num_sets = 0, frac_bits = 0, device = 0;
  unsigned char* d_kimg = nullptr;   // BF16 images (N = 64, 256)
  unsigned char* d_kimg8 = nullptr;  // E4M3 images (N = 64, 256)
  float* d_kscale = nullptr;         // E4M3 scale per set
  int16_t* d_kint = nullptr;         // round(2^f K)
};

// Round-to-nearest-even FP32 -> BF16 (finite inputs).
static uint16_t to_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

hygt_status dense_klt_create(dense_klt* out, int log2n, int num_sets, const float* h_K,
                             int frac_bits) {
  if (!out) return HYGT_ERR_ARG;
  *out = nullptr;
  if (!h_K || num_sets < 1 || num_sets > 65535 || frac_bits < 1 || frac_bits > 14)
    return HYGT_ERR_ARG;
  if (log2n != 4 && log2n != 6 && log2n != 8) return HYGT_ERR_UNSUPPORTED;
  const int N = 1 << log2n;
  const size_t per = (size_t)N * N;
  std::vector<int16_t> kint(per * num_sets);
  for (size_t i = 0; i < per * num_sets; ++i) {
    const double v = std::ldexp((double)h_K[i], frac_bits);
    if (!std::isfinite(v) || std::fabs(v) > 32767.0) return HYGT_ERR_ARG;
    kint[i] = (int16_t)std::lround(v);
  }
  // BF16 image: per 64-column K block, N rows of 128 bytes, 8-row groups of
  // 1024 bytes, 16-byte chunk c of row i stored at chunk c ^ (i % 8).
  std::vector<uint16_t> img;
  if (N >= 64) {
    img.assign(per * num_sets, 0);
    for (int s = 0; s < num_sets; ++s) {
      uint16_t* base = img.data() + (size_t)s * per;
      for (int kb = 0; kb < N / 64; ++kb)
        for (int i = 0; i < N; ++i)
          for (int c = 0; c < 8; ++c)
            for (int e = 0; e < 8; ++e) {
              const int k = kb * 64 + c * 8 + e;
              const size_t byte = (size_t)kb * N * 128 + (size_t)(i / 8) * 1024 +
                                  (size_t)(i % 8) * 128 + (size_t)((c ^ (i % 8)) * 16) + 2 * e;
              base[byte / 2] = to_bf16(h_K[(size_t)s * per + (size_t)i * N + k]);
            }
    }
  }
  // E4M3 image: each set's matrix scaled by 448 / max|K| (its scale is
  // max|K| / 448), K padded with zeros to rows of KP = max(N, 128) bytes; per
  // 128-column K block, N rows of 128 bytes, 8-row groups of 1024 bytes,
  // 16-byte chunk c of row i stored at chunk c ^ (i % 8).
  std::vector<uint8_t> img8;
  std::vector<float> kscale;
  if (N >= 64) {
    const int KP = N < 128 ? 128 : N;
    img8.assign((size_t)N * KP * num_sets, 0);
    kscale.assign(num_sets, 1.f);
    for (int s = 0; s < num_sets; ++s) {
      const float* K = h_K + (size_t)s * per;
      float amax = 0.f;
      for (size_t i = 0; i < per; ++i) amax = std::max(amax, std::fabs(K[i]));
      const float inv = amax > 0.f ? 448.f / amax : 1.f;
      kscale[s] = amax > 0.f ? amax / 448.f : 1.f;
      uint8_t* base = img8.data() + (size_t)s * N * KP;
      for (int kb = 0; kb < KP / 128; ++kb)
        for (int i = 0; i < N; ++i)
          for (int c = 0; c < 8; ++c)
            for (int e = 0; e < 16; ++e) {
              const int k = kb * 128 + c * 16 + e;
              const size_t byte = (size_t)kb * N * 128 + (size_t)(i / 8) * 1024 +
                                  (size_t)(i % 8) * 128 + (size_t)((c ^ (i % 8)) * 16) + e;
              base[byte] = k < N ? (uint8_t)__nv_cvt_float_to_fp8(K[(size_t)i * N + k] * inv,
                                                                  __NV_SATFINITE, __NV_E4M3)
                                 : (uint8_t)0;
            }
    }
  }
  dense_klt d = new (std::nothrow) dense_klt_s();
  if (!d) return HYGT_ERR_OOM;
  d->log2n = log2n;
  d->num_sets = num_sets;
  d->frac_bits = frac_bits;
  if (cudaGetDevice(&d->device) != cudaSuccess) {
    delete d;
    return HYGT_ERR_CUDA;
  }
  hygt_status st = upload(reinterpret_cast<void**>(&d->d_kint), kint.data(), kint.size() * 2,
                          pad16(kint.size() * 2));
  if (st == HYGT_OK && !img.empty())
    st = upload(reinterpret_cast<void**>(&d->d_kimg), img.data(), img.size() * 2,
                pad16(img.size() * 2));
  if (st == HYGT_OK && !img8.empty())
    st = upload(reinterpret_cast<void**>(&d->d_kimg8), img8.data(), img8.size(),
                pad16(img8.size()));
  if (st == HYGT_OK && !kscale.empty())
    st = upload(reinterpret_cast<void**>(&d->d_kscale), kscale.data(), kscale.size() * 4,
                pad16(kscale.size() * 4));
  if (st != HYGT_OK) {
    dense_klt_destroy(d);
    return st;
  }
  *out = d;
  return HYGT_OK;
}

void dense_klt_destroy(dense_klt d) {
  if (!d) return;
  if (d->d_kimg) cudaFree(d->d_kimg);
  if (d->d_kimg8) cudaFree(d->d_kimg8);
  if (d->d_kscale) cudaFree(d->d_kscale);
  if (d->d_kint) cudaFree(d->d_kint);
  delete d;
}

size_t dense_klt_workspace_bytes(dense_klt d, int64_t nblocks) {
  if (!d || nblocks < 0 || nblocks > kBatchMaxBlocks) return 0;
  return hygt::batch_layout(d->num_sets, nblocks, 128).total;
}

hygt_status dense_klt_build(dense_klt d, const uint16_t* d_set, int64_t nblocks, void* d_work,
                            size_t work_bytes, hygt_stream stream) {
  if (!d || nblocks < 0 || nblocks > kBatchMaxBlocks || !d_work || !aligned16(d_work))
    return HYGT_ERR_ARG;
  if (work_bytes < hygt::batch_layout(d->num_sets, nblocks, 128).total) return HYGT_ERR_ARG;
  return to_status(hygt::batch_build(d_set, nblocks, d->num_sets, 128, d_work, (cudaStream_t)stream));
}

hygt_status dense_klt_apply(dense_klt d, const void* d_work, const int16_t* d_x, void* d_y,
                            int64_t nblocks, int kind, hygt_stream stream, int* d_status) {
  if (!d || nblocks < 0 || nblocks > kBatchMaxBlocks) return HYGT_ERR_ARG;
  if (nblocks == 0) return HYGT_OK;
  if (!d_work || !aligned16(d_work) || !d_x || !d_y || !aligned16(d_x) || !aligned16(d_y))
    return HYGT_ERR_ARG;
  if (kind != DENSE_KLT_BF16 && kind != DENSE_KLT_INT && kind != DENSE_KLT_FP8)
    return HYGT_ERR_ARG;
  if ((kind == DENSE_KLT_BF16 || kind == DENSE_KLT_FP8) && d->log2n < 6)
    return HYGT_ERR_UNSUPPORTED;
  if (kind == DENSE_KLT_INT && d->log2n > 6) return HYGT_ERR_UNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HYGT_ERR_CUDA;
  if (dev != d->device) return HYGT_ERR_ARG;
  const hygt::BatchLayout L = hygt::batch_layout(d->num_sets, nblocks, 128);
  const char* w = static_cast<const char*>(d_work);
  hygt::DenseParams p{};
  p.x = d_x;
  p.y = static_cast<float*>(d_y);
  p.yint = static_cast<int32_t*>(d_y);
  p.order = reinterpret_cast<const int*>(w + L.order);
  p.starts = reinterpret_cast<const int*>(w + L.starts);
  p.meta = reinterpret_cast<const int*>(w + L.meta);
  p.nblocks = nblocks;
  p.tmax = L.tmax;
  p.kimg = d->d_kimg;
  p.kimg8 = d->d_kimg8;
  p.kscale = d->d_kscale;
  p.kint = d->d_kint;
  p.num_sets = d->num_sets;
  p.frac_bits = d->frac_bits;
  p.status = d_status;
  return to_status(hygt::launch_dense(d->log2n, kind, p, (cudaStream_t)stream));
}

hygt_status hygt_plan_info(hygt_plan plan, int* log2n, int* rounds, int* num_sets, int* is_float) {
  if (!plan) return HYGT_ERR_ARG;
  if (log2n) *log2n = plan->log2n;
  if (rounds) *rounds = plan->rounds;
  if (num_sets) *num_sets = plan->num_sets;
  if (is_float) *is_float = plan->is_float;
  return HYGT_OK;
}

size_t hygt_param_bytes(int log2n, int rounds, int num_sets) {
  if (log2n < 1 || log2n > 16 || rounds < 1 || num_sets < 1) return 0;
  const size_t N = (size_t)1 << log2n;
  return (size_t)num_sets * (size_t)rounds * N * (size_t)log2n / 2;
}

const char* hygt_status_string(int status) {
  switch (status) {
    case HYGT_OK: return "ok";
    case HYGT_ERR_ARG: return "invalid argument";
    case HYGT_ERR_CUDA: return "CUDA runtime error";
    case HYGT_ERR_OOM: return "device allocation failed";
    case HYGT_ERR_SET_INDEX: return "set index out of range";
    case HYGT_ERR_UNSUPPORTED: return "operation not supported by this plan";
    case HYGT_ERR_TOO_LARGE: return "batch larger than the static scratch (8 MiB)";
    default: return "unknown status";
  }
}

}  // extern "C"

// ---------------------------------------------------------------- no allocation
// hygt_forward_static: the schedule lives in a file-scope device array
// instead of a caller workspace.  Host code cannot use the array's name as a
// device address (in host code it names a host-side stand-in), so every call
// looks the address up with cudaGetSymbolAddress, with the caller's device
// current.  The lookup is a host-side query once the module is loaded, and
// doing it per call (rather than caching one address per device index)
// stays right after a device reset, when the module is loaded again and the
// array may move.
namespace {

constexpr size_t kStaticScratchBytes = (size_t)8 << 20;
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

hygt_status static_scratch(void** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return HYGT_ERR_CUDA;
  }
  *out = p;
  return HYGT_OK;
}

}  // namespace

extern "C" hygt_status hygt_forward_static(hygt_plan plan, const int16_t* d_x, int32_t* d_y,
                                           const uint16_t* d_set, int64_t nblocks,
                                           hygt_stream stream, int* d_status) {
  hygt_status s = check_io(plan, d_x, d_y, nblocks);
  if (s != HYGT_OK || nblocks == 0) return s;
  if (plan->is_float) return HYGT_ERR_UNSUPPORTED;
  if (nblocks > kBatchMaxBlocks) return HYGT_ERR_TOO_LARGE;
  const int group = hygt::batch_group(plan->log2n);
  if (hygt_batch_workspace_bytes(plan, nblocks) > kStaticScratchBytes) return HYGT_ERR_TOO_LARGE;
  void* work = nullptr;
  s = static_scratch(&work);
  if (s != HYGT_OK) return s;
  cudaError_t e =
      hygt::batch_build(d_set, nblocks, plan->num_sets, group, work, (cudaStream_t)stream);
  if (e != cudaSuccess) return to_status(e);
  const hygt::BatchParams p = make_batch_params(plan, work, d_x, d_y, nblocks, d_status);
  return to_status(hygt::launch_batch_fwd(plan->log2n, p, (cudaStream_t)stream));
}
