// The dictionary sweep from host memory to host memory with the host-device copies overlapped
// (mrom_sweep_host): the objects are cut into contiguous groups of about equal cost, and the
// groups alternate between two library-owned streams, so that group c's upload, object creation
// and plan overlap group c - 1's kernels, and group c - 1's read-back overlaps group c's.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "mrom_internal.h"

namespace mrom {
namespace {

// Bytes of an object's region in a packed dictionary (the layout of mrom_packed_obj).
size_t packed_region_bytes(const mrom_packed_obj& o) {
  const size_t r = (size_t)o.r;
  size_t n = r * r * (2 + (o.has_kin ? 1 : 0) + (o.has_me ? 1 : 0)) + 3 * r;
  if (o.has_gram) n += (2 * r + 3) * (2 * r + 3);
  return n * 16;
}

// Relative cost of an object in a sweep over n_w frequencies (float64 flops of the pencil
// route's preparation and its O(r) sweep).
double object_cost(int r, int n_w) { return 60.0 * r * r * r + 130.0 * (double)n_w * r; }

}  // namespace
}  // namespace mrom

using namespace mrom;

extern "C" mrom_status mrom_sweep_host(mrom_handle h, int32_t n_obj, const mrom_packed_obj* objects,
                                       const void* packed, size_t bytes, const double* omega, int32_t n_w,
                                       double* R, double* I, double* Delta, int32_t n_chunks) {
  if (!h) return MROM_EINVAL;
  if (n_obj < 1 || n_obj > 65535 || !objects || !packed || !omega || n_w < 1 || !R || !I || n_chunks < 1 ||
      n_chunks > 16)
    return fail(h, MROM_EINVAL,
                "mrom_sweep_host: 1 <= n_obj <= 65535, n_w >= 1, 1 <= n_chunks <= 16 and non-null arguments required");
  for (int o = 0; o < n_obj; ++o) {
    const mrom_packed_obj& e = objects[o];
    if (e.r < 1 || e.r > MROM_MAX_R || e.offset < 0 || (size_t)e.offset + packed_region_bytes(e) > bytes)
      return fail(h, MROM_EINVAL, "mrom_sweep_host: object " + std::to_string(o) + " lies outside the buffer");
  }
  cudaError_t ce = cudaSetDevice(h->device);
  if (ce != cudaSuccess) return cuda_fail(h, ce, "cudaSetDevice");
  for (cudaStream_t& s : h->aux)
    if (!s) {
      ce = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
      if (ce != cudaSuccess) return cuda_fail(h, ce, "mrom_sweep_host: stream creation");
    }
  n_chunks = std::min<int>(n_chunks, n_obj);

  // contiguous groups of about equal cost
  std::vector<double> cum(n_obj + 1, 0.0);
  for (int o = 0; o < n_obj; ++o) cum[o + 1] = cum[o] + object_cost(objects[o].r, n_w);
  std::vector<int> first(n_chunks + 1, 0);
  first[n_chunks] = n_obj;
  for (int c = 1; c < n_chunks; ++c) {
    const double target = cum[n_obj] * c / n_chunks;
    int o = (int)(std::lower_bound(cum.begin(), cum.end(), target) - cum.begin());
    first[c] = std::min(std::max(o, first[c - 1] + 1), n_obj - (n_chunks - c));
  }

  const cudaStream_t user = h->stream;
  const size_t per_obj = (size_t)n_w * 9;
  const int n_out = Delta ? 3 : 2;
  double* d_buf = nullptr;  // omega, then R, I (and Delta) of every object
  ce = cudaMallocAsync(reinterpret_cast<void**>(&d_buf), ((size_t)n_w + n_out * per_obj * n_obj) * sizeof(double),
                       user);
  if (ce != cudaSuccess) return fail(h, MROM_ENOMEM, "mrom_sweep_host: device allocation failed");
  double* d_om = d_buf;
  double* d_out[3] = {d_buf + n_w, d_buf + n_w + per_obj * n_obj, Delta ? d_buf + n_w + 2 * per_obj * n_obj : nullptr};
  double* h_out[3] = {R, I, Delta};
  ce = cudaMemcpyAsync(d_om, omega, (size_t)n_w * sizeof(double), cudaMemcpyDefault, user);
  cudaEvent_t ready = nullptr;
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventRecord(ready, user);
  for (int k = 0; k < 2 && ce == cudaSuccess; ++k) ce = cudaStreamWaitEvent(h->aux[k], ready, 0);
  if (ce != cudaSuccess) {
    if (ready) cudaEventDestroy(ready);
    cudaFreeAsync(d_buf, user);
    return cuda_fail(h, ce, "mrom_sweep_host: setup");
  }

  std::vector<mrom_rom_t> roms(n_obj, nullptr);
  std::vector<mrom_plan> plans(n_chunks, nullptr);
  mrom_status st = MROM_OK;
  std::string msg;
  for (int c = 0; c < n_chunks && st == MROM_OK; ++c) {
    h->stream = h->aux[c & 1];
    const int o0 = first[c], n = first[c + 1] - first[c];
    // the group's part of the packed buffer, with offsets relative to its start (16-aligned)
    int64_t lo = objects[o0].offset, hi = 0;
    for (int o = o0; o < o0 + n; ++o) {
      lo = std::min<int64_t>(lo, objects[o].offset);
      hi = std::max<int64_t>(hi, objects[o].offset + (int64_t)packed_region_bytes(objects[o]));
    }
    lo = lo / 16 * 16;
    std::vector<mrom_packed_obj> recs(objects + o0, objects + o0 + n);
    for (auto& e : recs) e.offset -= lo;
    st = mrom_rom_from_packed(h, n, recs.data(), static_cast<const char*>(packed) + lo, (size_t)(hi - lo),
                              roms.data() + o0);
    if (st == MROM_OK) st = mrom_plan_create(h, roms.data() + o0, n, n_w, &plans[c]);
    if (st == MROM_OK)
      st = mrom_plan_sweep(plans[c], d_om, 0, d_out[0] + per_obj * o0, d_out[1] + per_obj * o0,
                           Delta ? d_out[2] + per_obj * o0 : nullptr);
    for (int q = 0; q < n_out && st == MROM_OK; ++q) {
      ce = cudaMemcpyAsync(h_out[q] + per_obj * o0, d_out[q] + per_obj * o0, per_obj * n * sizeof(double),
                           cudaMemcpyDefault, h->stream);
      if (ce != cudaSuccess) st = cuda_fail(h, ce, "mrom_sweep_host: read-back");
    }
    if (st != MROM_OK) msg = h->last_error;
  }
  // wait for both streams, then the device status of every group's sweep
  for (cudaStream_t s : h->aux) {
    ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess && st == MROM_OK) {
      st = cuda_fail(h, ce, "mrom_sweep_host");
      msg = h->last_error;
    }
  }
  h->stream = h->aux[0];
  if (st == MROM_OK) {
    st = mrom_synchronize(h);
    if (st != MROM_OK) msg = h->last_error;
  }
  for (mrom_plan p : plans)
    if (p) mrom_plan_destroy(p);
  mrom_rom_free_batch(roms.data(), n_obj);
  for (cudaStream_t s : h->aux) cudaStreamSynchronize(s);
  h->stream = user;
  cudaFreeAsync(d_buf, user);
  cudaEventDestroy(ready);
  if (st != MROM_OK) return fail(h, st, msg);
  return MROM_OK;
}
