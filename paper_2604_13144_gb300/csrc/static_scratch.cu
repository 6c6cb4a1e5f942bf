// tepai_sample_values_static: the ensemble run for callers that cannot
// allocate device memory themselves or through the library: a host that hands
// each component a fixed device budget and forbids further allocations, a
// plug-in that only receives buffers its framework allocated, or code that must
// not pay cudaMalloc's implicit device synchronisation on its path. All scratch
// of this entry point lives in one file-scope device array of fixed size; the
// caller passes the output buffers.
#include <cstring>
#include <mutex>

#include "host_plan.h"

namespace tepai {
cudaError_t launch_ensemble_f32(const KArgs& a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t launch_ensemble_f64(const KArgs& a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t occupancy_ensemble_f32(int block, size_t smem, int use_tc, int* ctas_per_sm);
cudaError_t occupancy_ensemble_f64(int block, size_t smem, int use_tc, int* ctas_per_sm);
}  // namespace tepai

using namespace tepai;

namespace {

// 64 MiB of scratch, held by every GPU that loads the library until the
// process exits. In host code `g_static_scratch` is only a host-side stand-in
// for the symbol: its device address comes from cudaGetSymbolAddress.
constexpr size_t kStaticScratchBytes = size_t(64) << 20;
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};
// Host-side plan of the call in flight, in static storage (no heap); guarded by
// g_static_mu for the whole call.
FixedPlan g_static_plan;

inline size_t a256(size_t x) { return (x + 255) / 256 * 256; }

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and kept for the life of the process.
// cudaDeviceReset unloads the module that holds the array, so the kept address
// is stale after it: a process that resets a device must not call this entry
// point again on that device.
int static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return TEPAI_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return TEPAI_ERR_INVALID_ARG;
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return TEPAI_ERR_CUDA;
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return TEPAI_OK;
}

}  // namespace

extern "C" int tepai_sample_values_static(const tepai_problem* P, const tepai_params* Q, double* d_v,
                                          signed char* d_sign, void* stream) {
  if (!d_v || !d_sign) return TEPAI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_static_mu);
  FixedPlan& hp = g_static_plan;
  int rc = build_plan(P, Q, hp);
  if (rc) return rc;
  if (Q->n_samples < 1) return TEPAI_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* base_v = nullptr;
  rc = static_scratch(&base_v);
  if (rc) return rc;
  char* base = static_cast<char*>(base_v);
  const int cap = Q->chi_max;
  const int csize = Q->precision == TEPAI_FP64 ? 16 : 8;
  // layout inside the static array: tables, counters, then per-CTA arenas
  size_t o = 0;
  const size_t o_terms = o; o = a256(o + sizeof(TermDev) * hp.L);
  const size_t o_snaps = o; o = a256(o + sizeof(int) * hp.M);
  const size_t o_obs = o; o = a256(o + sizeof(int) * hp.n_obs);
  const size_t o_bits = o; o = a256(o + hp.n);
  const size_t o_ops = o; o = a256(o + hp.obs_ops.size());
  const size_t o_stats = o; o = a256(o + sizeof(DevStats));
  const size_t o_counter = o; o = a256(o + sizeof(unsigned long long));
  const size_t o_status = o; o = a256(o + 4 * sizeof(int));
  const size_t o_arena = o;
  const size_t stride = a256(((size_t)hp.n * 2 * cap * cap + (Q->three_site ? 24 : 8) * (size_t)cap * cap) * csize);
  if (o_arena + stride > kStaticScratchBytes) return TEPAI_ERR_WORKSPACE_TOO_SMALL;
  // launch shape: the same rule as the allocating entry points
  int dev = 0, sms = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return TEPAI_ERR_CUDA;
  auto occ = [&](int blk, size_t sm_bytes, int use_tc, int* per) {
    return Q->precision == TEPAI_FP64 ? occupancy_ensemble_f64(blk, sm_bytes, use_tc, per)
                                      : occupancy_ensemble_f32(blk, sm_bytes, use_tc, per);
  };
  LaunchShape ls{};
  if (choose_launch_shape(hp.n, hp.L, Q->variant == TEPAI_CONTINUOUS ? hp.L : 0, cap, csize, optin, occ, ls, Q->launch_variant) != cudaSuccess)
    return TEPAI_ERR_CUDA;
  const int block = ls.block, x_elems = ls.x_elems, x_in_smem = ls.x_in_smem, per_sm = ls.per_sm;
  const size_t smem = ls.smem;
  long long grid = (long long)sms * (per_sm < 1 ? 1 : per_sm);
  const long long fit = (long long)((kStaticScratchBytes - o_arena) / stride);
  if (grid > fit) grid = fit;
  if (grid > Q->n_samples) grid = Q->n_samples;
  // tables (host -> static array) and the counters that must start at zero
  if (cudaMemcpyAsync(base + o_terms, hp.terms.data(), sizeof(TermDev) * hp.L, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(base + o_snaps, hp.snaps.data(), sizeof(int) * hp.M, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(base + o_obs, hp.obs.data(), sizeof(int) * hp.n_obs, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(base + o_bits, hp.bits.data(), hp.n, cudaMemcpyHostToDevice, st) ||
      (!hp.obs_ops.empty() &&
       cudaMemcpyAsync(base + o_ops, hp.obs_ops.data(), hp.obs_ops.size(), cudaMemcpyHostToDevice, st)) ||
      cudaMemsetAsync(base + o_stats, 0, o_arena - o_stats, st))
    return TEPAI_ERR_CUDA;
  KArgs a{};
  a.n = hp.n; a.L = hp.L; a.M = hp.M; a.n_obs = hp.n_obs; a.chi_cap = cap;
  a.periodic = hp.periodic; a.variant = Q->variant;
  const NumCfg nc = num_cfg(Q->precision);
  a.max_sweeps = nc.max_sweeps;
  a.N = hp.N; a.run_steps = hp.run_steps; a.n_samples = Q->n_samples; a.sample_offset = Q->sample_offset;
  a.seed = Q->seed; a.t_run = hp.t_run; a.cutoff = Q->cutoff;
  a.floor_rel = nc.floor_rel;
  a.tol = nc.tol;
  a.gap_rel = tie_band(Q);
  a.terms = reinterpret_cast<const TermDev*>(base + o_terms);
  a.snaps = reinterpret_cast<const int*>(base + o_snaps);
  a.obs = reinterpret_cast<const int*>(base + o_obs);
  a.init_bits = reinterpret_cast<const unsigned char*>(base + o_bits);
  a.obs_ops = hp.obs_ops.empty() ? nullptr : reinterpret_cast<const unsigned char*>(base + o_ops);
  a.arena = base + o_arena; a.arena_stride = stride;
  a.v = d_v; a.sign = d_sign;
  a.stats = reinterpret_cast<DevStats*>(base + o_stats);
  a.counter = reinterpret_cast<unsigned long long*>(base + o_counter);
  a.status = reinterpret_cast<int*>(base + o_status);
  a.x_in_smem = x_in_smem; a.smem_x_elems = x_elems; a.use_tc = ls.use_tc;
  a.precondition = jacobi_precondition();
  a.three_site = Q->three_site ? 1 : 0;
  const cudaError_t le = Q->precision == TEPAI_FP64 ? launch_ensemble_f64(a, (int)grid, block, smem, st)
                                                    : launch_ensemble_f32(a, (int)grid, block, smem, st);
  if (le != cudaSuccess) return TEPAI_ERR_CUDA;
  // the host tables above must outlive their asynchronous copies
  if (cudaStreamSynchronize(st) != cudaSuccess) return TEPAI_ERR_CUDA;
  int status = 0;
  if (cudaMemcpy(&status, base + o_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return TEPAI_ERR_CUDA;
  return status ? TEPAI_ERR_DEVICE_CHECK : TEPAI_OK;
}
