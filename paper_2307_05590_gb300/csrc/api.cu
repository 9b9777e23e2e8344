// Handles, plans and the sweep entry points of the C ABI.
#include "mrom_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <numeric>

namespace mrom {

mrom_status fail(mrom_ctx* h, mrom_status s, const std::string& msg) {
  if (h) h->last_error = msg;
  return s;
}

mrom_status cuda_fail(mrom_ctx* h, cudaError_t e, const char* what) {
  if (h) h->last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? MROM_ENOMEM : MROM_ECUDA;
}

}  // namespace mrom

using namespace mrom;

namespace {
constexpr uint64_t kPoolKeepBytes = 8ull << 30;  // freed stream-ordered memory kept for reuse
}  // namespace

extern "C" mrom_status mrom_create(int device, void* cuda_stream, mrom_handle* out) {
  if (!out) return MROM_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return MROM_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return MROM_ECUDA;
  auto* h = new mrom_ctx();
  h->device = device;
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  h->smem_optin = (size_t)optin;
  // NULL is CUDA's default stream, as everywhere in the runtime API
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  // The library's per-call blocks are stream-ordered allocations from the device's default pool.
  // With the pool's default release threshold (0) the memory goes back to the driver at every
  // synchronisation and is mapped again by the next call; keep up to kPoolKeepBytes cached in
  // this process instead (a process-local pool attribute, raised only if it is lower).
  {
    cudaMemPool_t pool = nullptr;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t cur = 0;
      if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur) == cudaSuccess && cur < kPoolKeepBytes) {
        uint64_t keep = kPoolKeepBytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      }
    }
    cudaGetLastError();
  }
  if (cudaMalloc(&h->d_status, sizeof(int)) != cudaSuccess ||
      cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    if (h->d_status) cudaFree(h->d_status);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
    return MROM_ENOMEM;
  }
  *out = h;
  return MROM_OK;
}

extern "C" mrom_status mrom_destroy(mrom_handle h) {
  if (!h) return MROM_EINVAL;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  for (cudaStream_t s : h->aux)
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  if (h->d_status) cudaFree(h->d_status);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  delete h;
  return MROM_OK;
}

extern "C" mrom_status mrom_set_stream(mrom_handle h, void* cuda_stream) {
  if (!h) return MROM_EINVAL;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  return MROM_OK;
}

extern "C" const char* mrom_last_error(mrom_handle h) {
  return h ? h->last_error.c_str() : "null handle";
}

extern "C" int64_t mrom_launch_count(mrom_handle h) { return h ? h->launches : 0; }

extern "C" mrom_status mrom_set_projection_precision(mrom_handle h, mrom_precision precision) {
  if (!h) return MROM_EINVAL;
  if (precision != MROM_FP64 && precision != MROM_MIXED)
    return fail(h, MROM_EINVAL, "mrom_set_projection_precision: MROM_FP64 or MROM_MIXED");
  h->projection_precision = precision;
  return MROM_OK;
}

extern "C" mrom_status mrom_synchronize(mrom_handle h) {
  if (!h) return MROM_EINVAL;
  cudaSetDevice(h->device);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_synchronize");
  int st = 0;
  e = cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_synchronize: status read");
  if (st) {
    cudaMemset(h->d_status, 0, sizeof(int));
    if (st & kStatusBadOmega) return fail(h, MROM_EINVAL, "a frequency was non-finite or <= 0");
    if (st & kStatusSingular) return fail(h, MROM_ESINGULAR, "zero or non-finite pivot in a reduced solve");
    if (st & kStatusTimeout) return fail(h, MROM_ETIMEOUT, "a bounded device wait gave up");
    if (st & kStatusConfig) return fail(h, MROM_ECUDA, "internal: a kernel launch had too little shared memory");
  }
  mrom_status p = h->pending;
  h->pending = MROM_OK;
  return p;
}

// ------------------------------------------------------------------ plans

namespace {



// Dynamic shared memory per CTA: an SM's shared memory divided by the CTAs that
// co-reside, so that they fill each other's barrier waits (minus the reservation).
size_t sweep_budget(const mrom_ctx* h, int cfg) {
  int per_sm = 0;
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device);
  const size_t share = (size_t)per_sm / sweep_fp64_ctas_per_sm(cfg);
  return std::min<size_t>(h->smem_optin, share) - 2048;
}

int default_config(const mrom_ctx* h) {
  if (h->sweep_cfg >= 0) return h->sweep_cfg;
  const char* env = std::getenv("MROM_SWEEP_CONFIG");
  if (env) {
    const int c = std::atoi(env);
    if (c >= 0 && c < sweep_fp64_num_configs()) return c;
  }
  return 1;  // 128 threads x 4 CTAs per SM: fastest on the 8..96 dictionary mix
}

}  // namespace

namespace mrom {

size_t sweep_budget_bytes(const mrom_ctx* h, int cfg) { return sweep_budget(h, cfg); }

int sweep_config(const mrom_ctx* h) { return default_config(h); }

RomDev rom_record(const mrom_rom* m) {
  RomDev d;
  d.K = m->K;
  d.Kin = m->has_kin ? m->Kin : nullptr;
  d.C = m->C;
  d.Me = m->Me;
  d.B = m->B;
  d.GKK = m->GKK;
  d.GCC = m->GCC;
  d.GSk = m->GSk;
  d.gsK = m->gsK;
  d.gsC = m->gsC;
  std::memcpy(d.gss, m->gss, sizeof(d.gss));
  std::memcpy(d.c00, m->c00, sizeof(d.c00));
  std::memcpy(d.N0, m->N0, sizeof(d.N0));
  d.alpha3 = m->alpha * m->alpha * m->alpha;
  d.cert_scale = m->has_cert ? d.alpha3 / (4.0 * m->alpha_lb) : 0.0;
  d.r = m->r;
  d.has_cert = m->has_cert ? 1 : 0;
  d.dB = nullptr;
  std::fill(d.dc00, d.dc00 + 9, 0.0);
  std::fill(d.dN0, d.dN0 + 9, 0.0);
  d.per_dir = (m->r_dirs[0] + m->r_dirs[1] + m->r_dirs[2]) > 0 ? 1 : 0;
  int off = 0;
  for (int i = 0; i < 3; ++i) {
    d.blk_lo[i] = d.per_dir ? off : 0;
    d.blk_hi[i] = d.per_dir ? off + m->r_dirs[i] : m->r;
    off += m->r_dirs[i];
  }
  return d;
}

// Pencil route of a plan: the LU kernel's task shapes for the routed table, then the tables.
mrom_status plan_pencil(mrom_ctx* h, mrom_plan plan, const std::vector<RomDev>& objs, size_t lu_budget) {
  const int n_obj = plan->n_obj, n_w = plan->n_w;
  std::vector<int> order_lu(n_obj);
  std::iota(order_lu.begin(), order_lu.end(), 0);
  std::stable_sort(order_lu.begin(), order_lu.end(), [&](int a, int b) { return objs[a].r > objs[b].r; });
  std::vector<int2> lu_info(n_obj);
  for (int k = 0; k < n_obj; ++k) {
    const int r = objs[order_lu[k]].r;
    const size_t per_s = sweep_fp64_bytes_per_system(r, true);
    const bool in_smem = per_s <= lu_budget;
    const int S = in_smem ? std::max(1, std::min<int>(n_w, (int)(lu_budget / per_s))) : 1;
    lu_info[k] = make_int2(S, in_smem ? 0 : 1);
  }
  return pencil_tables_create(h, objs, n_w, true, false, order_lu, lu_info, &plan->pen);
}

}  // namespace mrom

extern "C" mrom_status mrom_plan_create(mrom_handle h, const mrom_rom_t* roms, int32_t n_obj, int32_t n_w,
                                        mrom_plan* out) {
  if (!h) return MROM_EINVAL;
  if (!roms || !out || n_obj < 1 || n_w < 1) return fail(h, MROM_EINVAL, "mrom_plan_create: bad arguments");
  *out = nullptr;
  for (int o = 0; o < n_obj; ++o)
    if (!roms[o] || roms[o]->ctx != h) return fail(h, MROM_EINVAL, "mrom_plan_create: invalid object");
  cudaSetDevice(h->device);
  const int cfg = default_config(h);
  const size_t budget = sweep_budget(h, cfg);
  std::vector<RomDev> objs(n_obj);
  std::vector<SweepTask> tasks;
  std::vector<double> cost;
  bool all_cert = true;
  size_t smem = 0, ws_elems = 0;
  int64_t n_tasks_all = 0;
  // with pencil-route objects the LU kernel runs over the device-routed table, so the
  // explicit task list is only built for a plan that is LU throughout
  bool any_pencil = false;
  for (int o = 0; o < n_obj && h->solver == MROM_SOLVER_AUTO; ++o)
    any_pencil = any_pencil || (roms[o]->r_dirs[0] + roms[o]->r_dirs[1] + roms[o]->r_dirs[2]) == 0;
  for (int o = 0; o < n_obj; ++o) {
    const mrom_rom* m = roms[o];
    objs[o] = rom_record(m);
    all_cert = all_cert && m->has_cert;
    // matrices in shared memory when at least one system fits the budget, otherwise
    // in the CTA's slice of an L2-resident global workspace (one system per task)
    const size_t per_s = sweep_fp64_bytes_per_system(m->r, true);
    const bool in_smem = per_s <= budget;
    const size_t per = in_smem ? per_s : sweep_fp64_bytes_per_system(m->r, false);
    const int S = in_smem ? std::min<int>(n_w, (int)(budget / per_s)) : 1;
    if (!in_smem) ws_elems = std::max(ws_elems, sweep_fp64_matrix_elems(m->r));
    smem = std::max(smem, per * std::min(S, n_w));
    n_tasks_all += (n_w + S - 1) / S;
    if (any_pencil) continue;
    const double r = m->r;
    const double unit = 4.0 * r * r * r / 3.0 + 30.0 * r * r;
    for (int w0 = 0; w0 < n_w; w0 += S) {
      const int nw = std::min(S, n_w - w0);
      tasks.push_back(SweepTask{o, w0, nw, in_smem ? 0 : 1});
      cost.push_back(unit * nw);
    }
  }
  // longest tasks first: CTAs pull from the front of the list
  std::vector<int> order(tasks.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<SweepTask> sorted(tasks.size());
  for (size_t k = 0; k < order.size(); ++k) sorted[k] = tasks[order[k]];

  auto* plan = new mrom_plan_s();
  plan->ctx = h;
  plan->cfg = cfg;
  plan->n_obj = n_obj;
  plan->n_w = n_w;
  plan->all_cert = all_cert;
  plan->smem_bytes = smem;
  plan->n_tasks = (int)sorted.size();
  cudaError_t e = sweep_fp64_configure(cfg, smem);
  int occ = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sweep_fp64_symbol(cfg), sweep_fp64_threads(cfg), smem);
  occ = std::max(occ, 1);
  plan->grid = (int)std::min<int64_t>(n_tasks_all, (int64_t)h->num_sms * occ);
  plan->ws_elems = ws_elems;
  const size_t ws_bytes = ws_elems * sizeof(double2) * (size_t)plan->grid;
  const size_t bytes = ws_bytes + n_obj * sizeof(RomDev) + sorted.size() * sizeof(SweepTask) + 16;
  void* blk = nullptr;
  // stream-ordered allocation: the plan's tables are freed with cudaFreeAsync, so a
  // one-shot mrom_sweep never blocks the host
  if (e == cudaSuccess) e = cudaMallocAsync(&blk, bytes, h->stream);
  if (e != cudaSuccess) {
    delete plan;
    return cuda_fail(h, e, "mrom_plan_create");
  }
  plan->d_workspace = ws_elems ? static_cast<double2*>(blk) : nullptr;
  plan->d_objs = reinterpret_cast<RomDev*>(static_cast<char*>(blk) + ws_bytes);
  plan->d_tasks = reinterpret_cast<SweepTask*>(plan->d_objs + n_obj);
  plan->d_counter = reinterpret_cast<int*>(plan->d_tasks + sorted.size());
  e = cudaMemcpyAsync(plan->d_objs, objs.data(), n_obj * sizeof(RomDev), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(plan->d_tasks, sorted.data(), sorted.size() * sizeof(SweepTask),
                        cudaMemcpyHostToDevice, h->stream);
  // (copies from pageable host memory return once the source has been staged)
  if (e != cudaSuccess) {
    cudaFreeAsync(blk, h->stream);
    delete plan;
    return cuda_fail(h, e, "mrom_plan_create: upload");
  }
  if (h->solver == MROM_SOLVER_AUTO) {
    const mrom_status ps = plan_pencil(h, plan, objs, budget);
    if (ps != MROM_OK) {
      mrom_plan_destroy(plan);
      return ps;
    }
  }
  *out = plan;
  return MROM_OK;
}

extern "C" mrom_status mrom_plan_destroy(mrom_plan plan) {
  if (!plan) return MROM_EINVAL;
  cudaSetDevice(plan->ctx->device);
  pencil_tables_destroy(&plan->pen, plan->ctx->stream);
  for (auto& ev : plan->ev)
    if (ev) cudaEventDestroy(ev);
  cudaFreeAsync(plan->d_workspace ? static_cast<void*>(plan->d_workspace) : static_cast<void*>(plan->d_objs),
                plan->ctx->stream);
  delete plan;
  return MROM_OK;
}

namespace {

mrom_status run_plan(mrom_plan plan, const double* omega, int32_t omega_stride, const double* s_sigma,
                     double* R, double* I, double* Delta, double* eig = nullptr) {
  mrom_ctx* h = plan->ctx;
  if (!omega) return fail(h, MROM_EINVAL, "sweep: omega is null");
  if (omega_stride != 0 && omega_stride < plan->n_w)
    return fail(h, MROM_EINVAL, "sweep: omega_stride must be 0 or >= n_w");
  if (Delta && !plan->all_cert)
    return fail(h, MROM_EINVAL, "sweep: Delta requested but an object has no Gram matrix");
  if (!R && !I && !Delta && !eig) return MROM_OK;
  cudaSetDevice(h->device);
  auto mark = [&](int k) {
    if (plan->timing) cudaEventRecord(plan->ev[k], h->stream);
  };
  if (plan->pen.n_pen > 0) {
    // pencil route: per-object preparation and device-side routing, then both sweep kernels
    // (each over its own table; an empty table ends the kernel at once)
    const PencilTables& t = plan->pen;
    mark(0);
    cudaError_t e = pencil_tables_prepare(h, t, plan->d_objs, omega, omega_stride, s_sigma, nullptr);
    mark(1);
    if (e == cudaSuccess) e = pencil_tables_route(h, t);
    mark(2);
    if (e == cudaSuccess)
      e = launch_pencil_sweep(plan->d_objs, t.d_pens, t.d_table_pen, t.d_counters + 2, omega, omega_stride, s_sigma,
                              R, I, Delta, eig, h->d_status, plan->n_w, t.pen_grid, t.pen_smem, h->stream);
    mark(3);
    if (e == cudaSuccess)
      e = launch_sweep_fp64_routed(plan->cfg, plan->d_objs, t.d_table_lu, t.d_counters + 3, omega, omega_stride,
                                   s_sigma, R, I, Delta, eig, h->d_status, plan->n_w, plan->grid, plan->smem_bytes,
                                   plan->d_workspace, plan->ws_elems, h->stream);
    mark(4);
    if (e != cudaSuccess) return cuda_fail(h, e, "sweep launch");
    h->launches += 2;
    return MROM_OK;
  }
  mark(0);
  mark(1);
  mark(2);
  mark(3);
  cudaError_t e = sweep_fp64_configure(plan->cfg, plan->smem_bytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(plan->d_counter, 0, sizeof(int), h->stream);
  if (e == cudaSuccess)
    e = launch_sweep_fp64(plan->cfg, plan->d_objs, plan->d_tasks, plan->n_tasks, plan->d_counter, omega, omega_stride,
                          s_sigma, R, I, Delta, eig, h->d_status, plan->n_w, plan->grid, plan->smem_bytes,
                          plan->d_workspace, plan->ws_elems, h->stream);
  mark(4);
  if (e != cudaSuccess) return cuda_fail(h, e, "sweep launch");
  ++h->launches;
  return MROM_OK;
}

}  // namespace

extern "C" mrom_status mrom_plan_solver_counts(mrom_plan plan, int32_t* n_pencil, int32_t* n_lu) {
  if (!plan) return MROM_EINVAL;
  mrom_ctx* h = plan->ctx;
  int c[2] = {0, plan->n_obj};
  if (plan->pen.n_pen > 0) {
    cudaSetDevice(h->device);
    cudaError_t e = cudaMemcpyAsync(c, plan->pen.d_counters + 4, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "mrom_plan_solver_counts");
  }
  if (n_pencil) *n_pencil = c[0];
  if (n_lu) *n_lu = c[1];
  return MROM_OK;
}

extern "C" mrom_status mrom_plan_timing(mrom_plan plan, int32_t enable, float* stage_ms) {
  if (!plan) return MROM_EINVAL;
  mrom_ctx* h = plan->ctx;
  cudaSetDevice(h->device);
  if (enable && !plan->timing) {
    for (auto& ev : plan->ev) {
      const cudaError_t e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return cuda_fail(h, e, "mrom_plan_timing: event");
    }
    plan->timing = true;
    return MROM_OK;
  }
  if (!stage_ms) return MROM_OK;
  if (!plan->timing) return fail(h, MROM_EINVAL, "mrom_plan_timing: timing is not enabled");
  cudaError_t e = cudaEventSynchronize(plan->ev[4]);
  for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventElapsedTime(&stage_ms[k], plan->ev[k], plan->ev[k + 1]);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_plan_timing: elapsed time");
  return MROM_OK;
}

extern "C" mrom_status mrom_set_solver(mrom_handle h, mrom_solver solver) {
  if (!h) return MROM_EINVAL;
  if (solver != MROM_SOLVER_AUTO && solver != MROM_SOLVER_LU)
    return fail(h, MROM_EINVAL, "mrom_set_solver: MROM_SOLVER_AUTO or MROM_SOLVER_LU");
  h->solver = solver;
  return MROM_OK;
}

extern "C" mrom_status mrom_plan_sweep(mrom_plan plan, const double* omega, int32_t omega_stride, double* R,
                                       double* I, double* Delta) {
  if (!plan) return MROM_EINVAL;
  return run_plan(plan, omega, omega_stride, nullptr, R, I, Delta);
}

extern "C" mrom_status mrom_plan_sweep_invariants(mrom_plan plan, const double* omega, int32_t omega_stride,
                                                  double* R, double* I, double* Delta, double* eig) {
  if (!plan) return MROM_EINVAL;
  return run_plan(plan, omega, omega_stride, nullptr, R, I, Delta, eig);
}

namespace mrom {
namespace {

// A plan's objects at per-object permeability scales s_mu: K(s) = K + (1/s - 1) K_in of every
// object into per-call buffers (the plan's sweeps then read K(s) as their K, and the pencil
// preparation runs unscaled), and for objects with a reduced static problem B(s), c00(s), N0(s)
// and, when the certificate is wanted, its Gram blocks at s.  *block receives the per-call
// allocation (freed by the caller after the sweep, stream-ordered).
mrom_status instantiate_scales(mrom_plan plan, const mrom_rom_t* roms, const double* s_mu, bool cert,
                               void** block) {
  mrom_ctx* h = plan->ctx;
  const int n_obj = plan->n_obj;
  cudaStream_t st = h->stream;
  size_t elems = 0;
  int m_max = 0, rmax = 1;
  for (int o = 0; o < n_obj; ++o) {
    const size_t r = roms[o]->r, m = roms[o]->mu.m;
    elems += r * r;
    rmax = std::max(rmax, (int)r);
    if (m > 0) {
      elems += 3 * r + 3 * m + (cert ? 2 * r * r + 6 * r : 0);
      m_max = std::max(m_max, (int)m);
    }
  }
  const size_t b_mus = (n_obj * sizeof(MuDev) + 255) / 256 * 256, b_jobs = (n_obj * sizeof(ScaleKJob) + 255) / 256 * 256;
  void* blk = nullptr;
  cudaError_t e = cudaMallocAsync(&blk, b_mus + b_jobs + elems * sizeof(double2), st);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_sweep: allocation");
  *block = blk;
  auto* d_mus = static_cast<MuDev*>(blk);
  auto* d_jobs = reinterpret_cast<ScaleKJob*>(static_cast<char*>(blk) + b_mus);
  auto* q = reinterpret_cast<double2*>(static_cast<char*>(blk) + b_mus + b_jobs);
  std::vector<MuDev> mus(n_obj);
  std::vector<ScaleKJob> jobs(n_obj);
  std::vector<RomDev> recs(n_obj);
  for (int o = 0; o < n_obj; ++o) {
    const mrom_rom* m = roms[o];
    const size_t r = m->r, mm = m->mu.m;
    recs[o] = rom_record(m);
    jobs[o] = ScaleKJob{m->K, m->Kin, q, (int)r, 0};
    recs[o].K = q;
    q += r * r;
    if (mm > 0) {
      mus[o] = m->mu;
      mus[o].Bdst = q; q += 3 * r;
      mus[o].ydst = q; q += 3 * mm;
      mus[o].dBdst = nullptr;
      recs[o].B = mus[o].Bdst;
      if (cert) {
        mus[o].GKKdst = q; q += r * r;
        mus[o].GSkdst = q; q += r * r;
        mus[o].gsKdst = q; q += 3 * r;
        mus[o].gsCdst = q; q += 3 * r;
        recs[o].GKK = mus[o].GKKdst;
        recs[o].GSk = mus[o].GSkdst;
        recs[o].gsK = mus[o].gsKdst;
        recs[o].gsC = mus[o].gsCdst;
      } else {
        mus[o].Gext = nullptr;
      }
    }
  }
  e = cudaMemcpyAsync(d_mus, mus.data(), n_obj * sizeof(MuDev), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_jobs, jobs.data(), n_obj * sizeof(ScaleKJob), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(plan->d_objs, recs.data(), n_obj * sizeof(RomDev), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_scale_k(d_jobs, n_obj, rmax, s_mu, st);
  if (e == cudaSuccess && m_max > 0) e = launch_mu_instance(d_mus, n_obj, m_max, s_mu, false, plan->d_objs, nullptr,
                                                            h->d_status, st);
  if (e == cudaSuccess && m_max > 0 && cert) e = launch_mu_cert(d_mus, n_obj, s_mu, plan->d_objs, st);
  h->launches += 1 + (m_max > 0 ? 1 + (cert ? 1 : 0) : 0);
  // (pageable host vectors: each copy has consumed its source on return)
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_sweep: scales");
  return MROM_OK;
}

}  // namespace
}  // namespace mrom

extern "C" mrom_status mrom_sweep(mrom_handle h, const mrom_rom_t* roms, int32_t n_obj, const double* omega,
                                  int32_t n_w, int32_t omega_stride, const double* s_sigma, const double* s_mu,
                                  double* R, double* I, double* Delta) {
  if (!h) return MROM_EINVAL;
  if (s_mu) {
    if (!roms || n_obj < 1) return fail(h, MROM_EINVAL, "mrom_sweep: bad arguments");
    for (int o = 0; o < n_obj; ++o) {
      if (!roms[o] || !roms[o]->has_kin) return fail(h, MROM_EINVAL, "mrom_sweep: s_mu needs K_in on every object");
      if (Delta && !roms[o]->mu.Gext)
        return fail(h, MROM_ENOTSUP, "mrom_sweep: the certificate at s_mu needs objects from mrom_project_mu "
                                     "with a certificate inner product");
    }
  }
  mrom_plan plan = nullptr;
  mrom_status st = mrom_plan_create(h, roms, n_obj, n_w, &plan);
  if (st != MROM_OK) return st;
  void* inst = nullptr;
  if (s_mu) st = instantiate_scales(plan, roms, s_mu, Delta != nullptr, &inst);
  if (st == MROM_OK) st = run_plan(plan, omega, omega_stride, s_sigma, R, I, Delta);
  if (inst) cudaFreeAsync(inst, h->stream);
  mrom_plan_destroy(plan);
  return st;
}

extern "C" mrom_status mrom_certificate(mrom_handle h, const mrom_rom_t* roms, int32_t n_obj,
                                        const double* omega, int32_t n_w, int32_t omega_stride, double* Delta) {
  if (!h) return MROM_EINVAL;
  if (!Delta) return fail(h, MROM_EINVAL, "mrom_certificate: Delta is null");
  return mrom_sweep(h, roms, n_obj, omega, n_w, omega_stride, nullptr, nullptr, nullptr, nullptr, Delta);
}

extern "C" mrom_status mrom_tune_pencil(mrom_handle h, const mrom_rom_t* roms, int32_t n_obj, int32_t n_w,
                                        int32_t* groups) {
  if (!h) return MROM_EINVAL;
  if (!roms || n_obj < 1 || n_w < 1) return fail(h, MROM_EINVAL, "mrom_tune_pencil: bad arguments");
  for (int o = 0; o < n_obj; ++o)
    if (!roms[o] || roms[o]->ctx != h) return fail(h, MROM_EINVAL, "mrom_tune_pencil: invalid object");
  cudaSetDevice(h->device);
  // a sample spread over the batch: up to 2000 objects and 2048 frequencies (the sweep's balance
  // over the SMs depends on the batch, so a small sample can prefer a mapping that loses on the
  // whole batch)
  const int ns = std::min<int>(n_obj, 2000), nw = std::min<int>(n_w, 2048);
  std::vector<mrom_rom_t> sample(ns);
  for (int k = 0; k < ns; ++k) sample[k] = roms[(int64_t)k * n_obj / ns];
  std::vector<double> om(nw);
  for (int k = 0; k < nw; ++k) om[k] = std::pow(10.0, 1.0 + 7.0 * k / std::max(1, nw - 1));
  const size_t out = (size_t)ns * nw * 9;
  double* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, (3 * out + nw) * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_tune_pencil: scratch allocation");
  double* d_om = buf + 3 * out;
  e = cudaMemcpyAsync(d_om, om.data(), nw * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  bool cert = true;
  for (auto* r : sample) cert = cert && r->has_cert;
  const int saved = h->pencil_fmax, saved_solver = h->solver;
  h->solver = MROM_SOLVER_AUTO;
  int best = -1;
  float best_ms = 0.f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int F = 8; F >= 1 && e == cudaSuccess; F /= 2) {
    h->pencil_fmax = F;
    mrom_plan plan = nullptr;
    if (mrom_plan_create(h, sample.data(), ns, nw, &plan) != MROM_OK) continue;
    mrom_plan_sweep(plan, d_om, 0, buf, buf + out, cert ? buf + 2 * out : nullptr);  // warm-up
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the faster of two
      cudaEventRecord(e0, h->stream);
      mrom_plan_sweep(plan, d_om, 0, buf, buf + out, cert ? buf + 2 * out : nullptr);
      cudaEventRecord(e1, h->stream);
      e = cudaEventSynchronize(e1);
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      ms = rep == 0 ? t : std::min(ms, t);
    }
    if (best < 0 || ms < best_ms) {
      best = F;
      best_ms = ms;
    }
    mrom_plan_destroy(plan);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(h->stream);
  cudaFree(buf);
  h->solver = saved_solver;
  if (e != cudaSuccess) {
    h->pencil_fmax = saved;
    return cuda_fail(h, e, "mrom_tune_pencil");
  }
  h->pencil_fmax = best < 0 ? saved : best;
  if (groups) *groups = h->pencil_fmax;
  return mrom_synchronize(h);
}

extern "C" mrom_status mrom_tune(mrom_handle h, const mrom_rom_t* roms, int32_t n_obj, int32_t n_w,
                                 int32_t* chosen) {
  if (!h) return MROM_EINVAL;
  if (!roms || n_obj < 1 || n_w < 1) return fail(h, MROM_EINVAL, "mrom_tune: bad arguments");
  cudaSetDevice(h->device);
  // a sample spread over the batch: up to 96 objects and 200 frequencies
  const int ns = std::min<int>(n_obj, 96), nw = std::min<int>(n_w, 200);
  std::vector<mrom_rom_t> sample(ns);
  for (int k = 0; k < ns; ++k) sample[k] = roms[(int64_t)k * n_obj / ns];
  std::vector<double> om(nw);
  for (int k = 0; k < nw; ++k) om[k] = std::pow(10.0, 1.0 + 7.0 * k / std::max(1, nw - 1));
  const size_t out = (size_t)ns * nw * 9;
  double* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, (3 * out + nw) * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_tune: scratch allocation");
  double* d_om = buf + 3 * out;
  e = cudaMemcpyAsync(d_om, om.data(), nw * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  bool cert = true;
  for (auto* r : sample) cert = cert && r->has_cert;
  const int saved = h->sweep_cfg;
  const int saved_solver = h->solver;
  h->solver = MROM_SOLVER_LU;  // the configurations are those of the LU kernel
  int best = -1;
  float best_ms = 0.f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int cfg = 0; cfg < sweep_fp64_num_configs() && e == cudaSuccess; ++cfg) {
    h->sweep_cfg = cfg;
    mrom_plan plan = nullptr;
    if (mrom_plan_create(h, sample.data(), ns, nw, &plan) != MROM_OK) continue;
    mrom_plan_sweep(plan, d_om, 0, buf, buf + out, cert ? buf + 2 * out : nullptr);  // warm-up
    cudaEventRecord(e0, h->stream);
    mrom_plan_sweep(plan, d_om, 0, buf, buf + out, cert ? buf + 2 * out : nullptr);
    cudaEventRecord(e1, h->stream);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best < 0 || ms < best_ms) {
      best = cfg;
      best_ms = ms;
    }
    mrom_plan_destroy(plan);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(h->stream);
  cudaFree(buf);
  h->solver = saved_solver;
  if (e != cudaSuccess) {
    h->sweep_cfg = saved;
    return cuda_fail(h, e, "mrom_tune");
  }
  h->sweep_cfg = best < 0 ? saved : best;
  if (chosen) *chosen = h->sweep_cfg;
  return MROM_OK;
}
