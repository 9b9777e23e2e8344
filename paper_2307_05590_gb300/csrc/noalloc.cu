// Allocation-free sweep (mrom_sweep_noalloc).
//
// Computes what mrom_sweep computes, for callers that cannot allocate device
// memory while they run.  Every piece of device scratch the sweep needs -- the
// object table, a compact task table, the work counter and the workspace of
// systems too large for shared memory -- lives in one fixed array of device
// memory declared in this file.  The host-side tables are built in host memory
// and copied in with cudaMemcpyAsync; nothing here calls cudaMalloc, cudaFree or
// any allocating routine.
#include "mrom_internal.h"

#include <algorithm>
#include <mutex>
#include <numeric>

namespace {

// The fixed scratch array.  Host code must not use this name as an address: on the
// host it is only a stand-in, so its device address is resolved once per device
// with cudaGetSymbolAddress (scratch_address below) and passed to the kernel.
static __device__ __align__(256) unsigned char g_sweep_scratch[MROM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_sweep_scratch on the handle's device (that device must be current).
mrom_status scratch_address(mrom_ctx* h, unsigned char** out) {
  if (h->device < 0 || h->device >= kMaxDevices)
    return mrom::fail(h, MROM_ENOTSUP, "mrom_sweep_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[h->device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sweep_scratch);
    if (e != cudaSuccess) return mrom::cuda_fail(h, e, "mrom_sweep_noalloc: cudaGetSymbolAddress");
    g_scratch_addr[h->device] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[h->device]);
  return MROM_OK;
}

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

using namespace mrom;

extern "C" mrom_status mrom_sweep_noalloc(mrom_handle h, const mrom_rom_t* roms, int32_t n_obj,
                                          const double* omega, int32_t n_w, int32_t omega_stride, double* R,
                                          double* I, double* Delta) {
  if (!h) return MROM_EINVAL;
  if (!roms || n_obj < 1 || n_w < 1 || !omega)
    return fail(h, MROM_EINVAL, "mrom_sweep_noalloc: bad arguments");
  if (omega_stride != 0 && omega_stride < n_w)
    return fail(h, MROM_EINVAL, "mrom_sweep_noalloc: omega_stride must be 0 or >= n_w");
  for (int o = 0; o < n_obj; ++o) {
    if (!roms[o] || roms[o]->ctx != h) return fail(h, MROM_EINVAL, "mrom_sweep_noalloc: invalid object");
    if (Delta && !roms[o]->has_cert)
      return fail(h, MROM_EINVAL, "mrom_sweep_noalloc: Delta requested but an object has no Gram matrix");
  }
  if (!R && !I && !Delta) return MROM_OK;
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_sweep_noalloc: cudaSetDevice");

  // ---- host-side tables (same task sizes as mrom_plan_create, objects in cost order)
  const int cfg = sweep_config(h);
  const size_t budget = sweep_budget_bytes(h, cfg);
  std::vector<int> S(n_obj), in_glob(n_obj), order(n_obj);
  std::vector<double> unit(n_obj);
  size_t smem = 0, ws_elems = 0;
  for (int o = 0; o < n_obj; ++o) {
    const int r = roms[o]->r;
    const size_t per_s = sweep_fp64_bytes_per_system(r, true);
    const bool in_smem = per_s <= budget;
    const size_t per = in_smem ? per_s : sweep_fp64_bytes_per_system(r, false);
    S[o] = in_smem ? std::min<int>(n_w, (int)(budget / per_s)) : 1;
    in_glob[o] = in_smem ? 0 : 1;
    if (!in_smem) ws_elems = std::max(ws_elems, sweep_fp64_matrix_elems(r));
    smem = std::max(smem, per * (size_t)S[o]);
    unit[o] = (4.0 * r * r * r / 3.0 + 30.0 * r * r) * S[o];
  }
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return unit[a] > unit[b]; });
  std::vector<SweepTask> table(n_obj + 1);
  table[0] = SweepTask{n_obj, 0, 0, 0};
  int64_t first = 0;
  for (int k = 0; k < n_obj; ++k) {
    const int o = order[k];
    table[k + 1] = SweepTask{o, (int)first, S[o], in_glob[o]};
    first += (n_w + S[o] - 1) / S[o];
    if (first > INT32_MAX) return fail(h, MROM_EINVAL, "mrom_sweep_noalloc: too many tasks");
  }
  const int n_tasks = (int)first;
  std::vector<RomDev> objs(n_obj);
  for (int o = 0; o < n_obj; ++o) objs[o] = rom_record(roms[o]);

  // ---- scratch layout: counter | object table | task table | workspace (grid slices)
  const size_t off_objs = 256;
  const size_t off_table = off_objs + round256(objs.size() * sizeof(RomDev));
  const size_t off_ws = off_table + round256(table.size() * sizeof(SweepTask));
  const size_t cap = (size_t)MROM_NOALLOC_SCRATCH_BYTES;
  const size_t ws_per_cta = ws_elems * sizeof(double2);
  if (off_ws + ws_per_cta > cap)
    return fail(h, MROM_EINVAL,
                "mrom_sweep_noalloc: batch needs " + std::to_string(off_ws + ws_per_cta) +
                    " bytes of scratch, more than the fixed MROM_NOALLOC_SCRATCH_BYTES = " + std::to_string(cap));
  // occupancy of the instantiation that is launched (the compact-table kernel)
  e = cudaFuncSetAttribute(sweep_fp64_implicit_symbol(cfg), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sweep_fp64_implicit_symbol(cfg), sweep_fp64_threads(cfg),
                                                      smem);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_sweep_noalloc: configuration");
  int grid = std::min(n_tasks, h->num_sms * std::max(occ, 1));
  if (ws_per_cta) grid = std::min<int64_t>(grid, (int64_t)((cap - off_ws) / ws_per_cta));

  unsigned char* base = nullptr;
  mrom_status st = scratch_address(h, &base);
  if (st != MROM_OK) return st;
  int* counter = reinterpret_cast<int*>(base);
  auto* d_objs = reinterpret_cast<RomDev*>(base + off_objs);
  auto* d_table = reinterpret_cast<SweepTask*>(base + off_table);
  auto* d_ws = ws_per_cta ? reinterpret_cast<double2*>(base + off_ws) : nullptr;

  // the array keeps the previous call's contents: the counter must start at zero
  e = cudaMemsetAsync(counter, 0, sizeof(int), h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_objs, objs.data(), objs.size() * sizeof(RomDev), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_table, table.data(), table.size() * sizeof(SweepTask), cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess)
    e = launch_sweep_fp64_implicit(cfg, d_objs, d_table, n_tasks, counter, omega, omega_stride, R, I, Delta,
                                   h->d_status, n_w, grid, smem, d_ws, ws_elems, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_sweep_noalloc: launch");
  ++h->launches;
  return MROM_OK;
}
