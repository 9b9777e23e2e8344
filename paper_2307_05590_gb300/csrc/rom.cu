// Reduced objects: device storage, input checks and the certificate Gram split.
#include "mrom_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

namespace mrom {
namespace {

// Split G (n x n, n = 2r+3, columns [C o_1, C o_2, C o_3 | (K+eps M)U | C U]) into the
// blocks the sweep kernel reads (Lemma 4.2; see sweep_fp64.cu for how they combine).
__global__ void split_gram_kernel(const double2* __restrict__ G, int r, double2* __restrict__ GKK,
                                  double2* __restrict__ GCC, double2* __restrict__ GSk,
                                  double2* __restrict__ gsK, double2* __restrict__ gsC) {
  const int n = 2 * r + 3;
  const int total = r * r;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total + 3 * r;
       idx += gridDim.x * blockDim.x) {
    if (idx < total) {
      const int a = idx / r, b = idx - (idx / r) * r;
      const int ka = 3 + a, kb = 3 + b, ca = 3 + r + a, cb = 3 + r + b;
      GKK[idx] = G[(size_t)ka * n + kb];
      GCC[idx] = G[(size_t)ca * n + cb];
      const double2 ck = G[(size_t)ca * n + kb], kc = G[(size_t)ka * n + cb];
      GSk[idx] = make_double2(ck.x - kc.x, ck.y - kc.y);
    } else {
      const int e = idx - total;
      const int i = e / r, a = e - (e / r) * r;
      gsK[e] = G[(size_t)i * n + 3 + a];
      gsC[e] = G[(size_t)i * n + 3 + r + a];
    }
  }
}

__global__ void nonfinite_kernel(const double* __restrict__ x, size_t n, int* __restrict__ flag) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) atomicOr(flag, 1);
}

}  // namespace

cudaError_t launch_split_gram(const double2* G, int r, double2* GKK, double2* GCC, double2* GSk,
                              double2* gsK, double2* gsC, cudaStream_t stream) {
  const int total = r * r + 3 * r;
  const int blocks = std::min(1024, (total + 255) / 256);
  split_gram_kernel<<<blocks, 256, 0, stream>>>(G, r, GKK, GCC, GSk, gsK, gsC);
  return cudaGetLastError();
}

cudaError_t launch_nonfinite(const double* x, size_t n, int* flag, cudaStream_t stream) {
  const int blocks = (int)std::min<size_t>(1024, (n + 255) / 256 + 1);
  nonfinite_kernel<<<blocks, 256, 0, stream>>>(x, n, flag);
  return cudaGetLastError();
}

}  // namespace mrom

using namespace mrom;

extern "C" mrom_status mrom_rom_from_reduced(mrom_handle h, const mrom_reduced_desc* d, mrom_rom_t* out) {
  if (!h) return MROM_EINVAL;
  if (!d || !out) return fail(h, MROM_EINVAL, "mrom_rom_from_reduced: null argument");
  *out = nullptr;
  const int r = d->r;
  if (r < 1 || r > MROM_MAX_R)
    return fail(h, MROM_EINVAL, "mrom_rom_from_reduced: r must be in [1, MROM_MAX_R]");
  if (!d->K || !d->C || !d->B || !d->c00)
    return fail(h, MROM_EINVAL, "mrom_rom_from_reduced: K, C, B and c00 are required");
  if (!std::isfinite(d->alpha) || !(d->alpha > 0) || !std::isfinite(d->vol_B))
    return fail(h, MROM_EINVAL, "mrom_rom_from_reduced: alpha must be finite and > 0");
  if (d->G && !(d->alpha_lb > 0 && std::isfinite(d->alpha_lb)))
    return fail(h, MROM_EINVAL, "mrom_rom_from_reduced: a Gram matrix needs alpha_lb > 0");
  const int rd_sum = d->r_dirs[0] + d->r_dirs[1] + d->r_dirs[2];
  if (rd_sum != 0 && (rd_sum != r || d->r_dirs[0] < 1 || d->r_dirs[1] < 1 || d->r_dirs[2] < 1))
    return fail(h, MROM_EINVAL, "mrom_rom_from_reduced: r_dirs must be all 0 or positive with sum r");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");

  const size_t rr = (size_t)r * r;
  const size_t ng = (size_t)(2 * r + 3);
  // layout: K, Kin, C, Me, B, G, GKK, GCC, GSk, gsK, gsC, flag
  size_t n2 = rr * 4 + 3 * (size_t)r + (d->G ? ng * ng + 3 * rr + 6 * (size_t)r : 0);
  void* block = nullptr;
  e = cudaMalloc(&block, n2 * sizeof(double2) + 16);
  if (e != cudaSuccess) return fail(h, MROM_ENOMEM, "mrom_rom_from_reduced: device allocation failed");
  auto* rom = new mrom_rom();
  rom->ctx = h;
  rom->r = r;
  rom->alpha = d->alpha;
  rom->alpha_lb = d->alpha_lb;
  rom->vol_B = d->vol_B;
  rom->d_block = block;
  double2* p = static_cast<double2*>(block);
  rom->K = p; p += rr;
  rom->Kin = p; p += rr;
  rom->C = p; p += rr;
  rom->Me = p; p += rr;
  rom->B = p; p += 3 * (size_t)r;
  if (d->G) {
    rom->G = p; p += ng * ng;
    rom->GKK = p; p += rr;
    rom->GCC = p; p += rr;
    rom->GSk = p; p += rr;
    rom->gsK = p; p += 3 * (size_t)r;
    rom->gsC = p; p += 3 * (size_t)r;
  }
  int* d_flag = reinterpret_cast<int*>(p);
  cudaStream_t st = h->stream;
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st);
  };
  e = cudaMemsetAsync(block, 0, n2 * sizeof(double2) + 16, st);
  cp(rom->K, d->K, rr * 16);
  if (d->K_in) cp(rom->Kin, d->K_in, rr * 16);
  cp(rom->C, d->C, rr * 16);
  if (d->Me) cp(rom->Me, d->Me, rr * 16);
  cp(rom->B, d->B, 3 * (size_t)r * 16);
  if (d->G) cp(rom->G, d->G, ng * ng * 16);
  double host9[9];
  if (e == cudaSuccess) e = cudaMemcpy(host9, d->c00, sizeof(host9), cudaMemcpyDefault);
  std::memcpy(rom->c00, host9, sizeof(host9));
  if (d->N0 && e == cudaSuccess) {
    e = cudaMemcpy(host9, d->N0, sizeof(host9), cudaMemcpyDefault);
    std::memcpy(rom->N0, host9, sizeof(host9));
  }
  if (e == cudaSuccess) e = launch_nonfinite(reinterpret_cast<const double*>(rom->K), 2 * n2, d_flag, st);
  if (e == cudaSuccess) ++h->launches;
  if (d->G && e == cudaSuccess) {
    e = launch_split_gram(rom->G, r, rom->GKK, rom->GCC, rom->GSk, rom->gsK, rom->gsC, st);
    if (e == cudaSuccess) ++h->launches;
  }
  int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    mrom_rom_free(rom);
    return cuda_fail(h, e, "mrom_rom_from_reduced");
  }
  bool bad = flag != 0;
  for (int k = 0; k < 9; ++k) bad = bad || !std::isfinite(rom->c00[k]) || !std::isfinite(rom->N0[k]);
  if (bad) {
    mrom_rom_free(rom);
    return fail(h, MROM_EINVAL, "mrom_rom_from_reduced: non-finite value in the reduced data");
  }
  if (d->G) {
    std::vector<double2> gss(9);
    for (int i = 0; i < 3; ++i) {
      e = cudaMemcpy(&gss[i * 3], rom->G + (size_t)i * ng, 3 * sizeof(double2), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        mrom_rom_free(rom);
        return cuda_fail(h, e, "mrom_rom_from_reduced: Gram read-back");
      }
    }
    for (int k = 0; k < 9; ++k) rom->gss[k] = gss[k].x;
    rom->has_cert = true;
  }
  rom->has_kin = d->K_in != nullptr;
  for (int i = 0; i < 3; ++i) rom->r_dirs[i] = d->r_dirs[i];
  if (!d->Me) rom->Me = nullptr;
  *out = rom;
  return MROM_OK;
}

extern "C" int32_t mrom_rom_rank(mrom_rom_t rom) { return rom ? rom->r : 0; }

extern "C" void mrom_rom_free_batch(mrom_rom_t* roms, int32_t n) {
  if (!roms) return;
  for (int32_t k = 0; k < n; ++k) {
    mrom_rom_free(roms[k]);
    roms[k] = nullptr;
  }
}

extern "C" void mrom_rom_free(mrom_rom_t rom) {
  if (!rom) return;
  if (rom->mu_block) cudaFree(rom->mu_block);
  if (rom->shared) {
    if (--rom->shared->refs == 0) {
      cudaFreeAsync(rom->shared->p, rom->shared->stream);
      delete rom->shared;
    }
  } else if (rom->d_block) {
    cudaFree(rom->d_block);
  }
  delete rom;
}

namespace mrom {
namespace {

// Per object: flag[o] = 1 when any of its len[o] doubles at seg[o] is not finite.
__global__ void nonfinite_batch_kernel(const double* const* __restrict__ seg, const size_t* __restrict__ len,
                                       int* __restrict__ flag) {
  const int o = blockIdx.y;
  const double* x = seg[o];
  const size_t n = len[o];
  int bad = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (bad) atomicOr(&flag[o], 1);
}

// gss[o][i][j] = Re G_o[i][j], i, j < 3 (the source-source block of the certificate Gram).
__global__ void gather_gss_kernel(const double2* const* __restrict__ G, const int* __restrict__ ng, int n,
                                  double* __restrict__ gss) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 9 * n; idx += gridDim.x * blockDim.x) {
    const int o = idx / 9, k = idx - (idx / 9) * 9;
    gss[idx] = G[o] ? G[o][(size_t)(k / 3) * ng[o] + (k % 3)].x : 0.0;
  }
}

// Gram split of many objects in one launch (blockIdx.y = object; objects without G skip).
struct SplitJob {
  const double2* G;
  double2 *GKK, *GCC, *GSk, *gsK, *gsC;
  int r, pad;
};

__global__ void split_gram_batch_kernel(const SplitJob* __restrict__ jobs) {
  const SplitJob j = jobs[blockIdx.y];
  if (!j.G) return;
  const int r = j.r, n = 2 * r + 3, total = r * r;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total + 3 * r; idx += gridDim.x * blockDim.x) {
    if (idx < total) {
      const int a = idx / r, b = idx - (idx / r) * r;
      const int ka = 3 + a, kb = 3 + b, ca = 3 + r + a, cb = 3 + r + b;
      j.GKK[idx] = j.G[(size_t)ka * n + kb];
      j.GCC[idx] = j.G[(size_t)ca * n + cb];
      const double2 ck = j.G[(size_t)ca * n + kb], kc = j.G[(size_t)ka * n + cb];
      j.GSk[idx] = make_double2(ck.x - kc.x, ck.y - kc.y);
    } else {
      const int e = idx - total;
      const int i = e / r, q = e - (e / r) * r;
      j.gsK[e] = j.G[(size_t)i * n + 3 + q];
      j.gsC[e] = j.G[(size_t)i * n + 3 + r + q];
    }
  }
}

mrom_status check_desc(mrom_ctx* h, const mrom_reduced_desc* d, const char* who) {
  const std::string w(who);
  const int r = d->r;
  if (r < 1 || r > MROM_MAX_R) return fail(h, MROM_EINVAL, w + ": r must be in [1, MROM_MAX_R]");
  if (!d->K || !d->C || !d->B || !d->c00) return fail(h, MROM_EINVAL, w + ": K, C, B and c00 are required");
  if (!std::isfinite(d->alpha) || !(d->alpha > 0) || !std::isfinite(d->vol_B))
    return fail(h, MROM_EINVAL, w + ": alpha must be finite and > 0");
  if (d->G && !(d->alpha_lb > 0 && std::isfinite(d->alpha_lb)))
    return fail(h, MROM_EINVAL, w + ": a Gram matrix needs alpha_lb > 0");
  const int rd_sum = d->r_dirs[0] + d->r_dirs[1] + d->r_dirs[2];
  if (rd_sum != 0 && (rd_sum != r || d->r_dirs[0] < 1 || d->r_dirs[1] < 1 || d->r_dirs[2] < 1))
    return fail(h, MROM_EINVAL, w + ": r_dirs must be all 0 or positive with sum r");
  return MROM_OK;
}

// 9 doubles from a host or device pointer
cudaError_t read9(const double* src, double* dst) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, src) == cudaSuccess && at.type == cudaMemoryTypeDevice)
    return cudaMemcpy(dst, src, 9 * sizeof(double), cudaMemcpyDeviceToHost);
  cudaGetLastError();  // clear a possible error from querying a plain host pointer
  std::memcpy(dst, src, 9 * sizeof(double));
  return cudaSuccess;
}

}  // namespace
}  // namespace mrom

extern "C" mrom_status mrom_rom_from_reduced_batch(mrom_handle h, int32_t n_obj, const mrom_reduced_desc* descs,
                                                   mrom_rom_t* out) {
  if (!h) return MROM_EINVAL;
  if (n_obj < 1 || n_obj > 65535 || !descs || !out)
    return fail(h, MROM_EINVAL, "mrom_rom_from_reduced_batch: 1 <= n_obj <= 65535 and non-null arrays required");
  for (int o = 0; o < n_obj; ++o) {
    out[o] = nullptr;
    const mrom_status st = check_desc(h, &descs[o], "mrom_rom_from_reduced_batch");
    if (st != MROM_OK) return fail(h, st, h->last_error + " (object " + std::to_string(o) + ")");
  }
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  cudaStream_t st = h->stream;
  // layout per object as in mrom_rom_from_reduced: K, Kin, C, Me, B, [G, GKK, GCC, GSk, gsK, gsC]
  std::vector<size_t> off(n_obj), cnt(n_obj);
  size_t total = 0;
  for (int o = 0; o < n_obj; ++o) {
    const size_t r = descs[o].r, rr = r * r, ng = 2 * r + 3;
    cnt[o] = rr * 4 + 3 * r + (descs[o].G ? ng * ng + 3 * rr + 6 * r : 0);
    off[o] = total;
    total += cnt[o];
  }
  // tail: per-object flags (int), gss (9 doubles), segment and Gram pointer tables
  const size_t b_data = total * sizeof(double2);
  const size_t b_flag = ((size_t)n_obj * sizeof(int) + 15) / 16 * 16;
  const size_t b_gss = (size_t)n_obj * 9 * sizeof(double);
  const size_t b_tab = (size_t)n_obj * (2 * sizeof(void*) + sizeof(size_t) + sizeof(int));
  void* block = nullptr;
  e = cudaMallocAsync(&block, b_data + b_flag + b_gss + b_tab + 64, st);
  if (e != cudaSuccess) return fail(h, MROM_ENOMEM, "mrom_rom_from_reduced_batch: device allocation failed");
  auto* shared = new mrom_rom::SharedBlock();
  shared->p = block;
  shared->stream = st;
  char* base = static_cast<char*>(block);
  int* d_flag = reinterpret_cast<int*>(base + b_data);
  double* d_gss = reinterpret_cast<double*>(base + b_data + b_flag);
  char* tab = base + b_data + b_flag + b_gss;
  tab = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(tab) + 15) / 16 * 16);
  auto** d_seg = reinterpret_cast<const double**>(tab);
  auto** d_g = reinterpret_cast<const double2**>(tab + (size_t)n_obj * sizeof(void*));
  auto* d_len = reinterpret_cast<size_t*>(tab + (size_t)n_obj * 2 * sizeof(void*));
  auto* d_ng = reinterpret_cast<int*>(tab + (size_t)n_obj * (2 * sizeof(void*) + sizeof(size_t)));

  std::vector<mrom_rom*> roms(n_obj, nullptr);
  std::vector<const double*> seg(n_obj);
  std::vector<const double2*> gp(n_obj);
  std::vector<size_t> len(n_obj);
  std::vector<int> ngv(n_obj);
  auto cleanup = [&](mrom_status s, const std::string& msg) {
    for (auto* m : roms) delete m;
    cudaFreeAsync(block, st);
    delete shared;
    return fail(h, s, msg);
  };
  e = cudaMemsetAsync(block, 0, b_data + b_flag, st);
  for (int o = 0; o < n_obj && e == cudaSuccess; ++o) {
    const mrom_reduced_desc* d = &descs[o];
    const size_t r = d->r, rr = r * r, ng = 2 * r + 3;
    auto* rom = new mrom_rom();
    roms[o] = rom;
    rom->ctx = h;
    rom->r = d->r;
    rom->alpha = d->alpha;
    rom->alpha_lb = d->alpha_lb;
    rom->vol_B = d->vol_B;
    rom->shared = shared;
    double2* p = static_cast<double2*>(block) + off[o];
    rom->K = p; p += rr;
    rom->Kin = p; p += rr;
    rom->C = p; p += rr;
    rom->Me = p; p += rr;
    rom->B = p; p += 3 * r;
    if (d->G) {
      rom->G = p; p += ng * ng;
      rom->GKK = p; p += rr;
      rom->GCC = p; p += rr;
      rom->GSk = p; p += rr;
      rom->gsK = p; p += 3 * r;
      rom->gsC = p; p += 3 * r;
    }
    auto cp = [&](void* dst, const void* src, size_t bytes) {
      if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st);
    };
    cp(rom->K, d->K, rr * 16);
    if (d->K_in) cp(rom->Kin, d->K_in, rr * 16);
    cp(rom->C, d->C, rr * 16);
    if (d->Me) cp(rom->Me, d->Me, rr * 16);
    cp(rom->B, d->B, 3 * r * 16);
    if (d->G) cp(rom->G, d->G, ng * ng * 16);
    if (e == cudaSuccess) e = read9(d->c00, rom->c00);
    if (e == cudaSuccess && d->N0) e = read9(d->N0, rom->N0);
    seg[o] = reinterpret_cast<const double*>(static_cast<double2*>(block) + off[o]);
    len[o] = 2 * cnt[o];
    gp[o] = rom->G;
    ngv[o] = (int)ng;
    rom->has_cert = d->G != nullptr;
    rom->has_kin = d->K_in != nullptr;
    for (int i = 0; i < 3; ++i) rom->r_dirs[i] = d->r_dirs[i];
    if (!d->Me) rom->Me = nullptr;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_seg, seg.data(), n_obj * sizeof(void*), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_g, gp.data(), n_obj * sizeof(void*), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_len, len.data(), n_obj * sizeof(size_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_ng, ngv.data(), n_obj * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cleanup(MROM_ECUDA, std::string("mrom_rom_from_reduced_batch: upload: ") +
                                                     cudaGetErrorString(e));
  // (the host staging vectors above are pageable: each copy has consumed its source on return)
  nonfinite_batch_kernel<<<dim3(8, (unsigned)n_obj), 256, 0, st>>>(d_seg, d_len, d_flag);
  gather_gss_kernel<<<std::max(1, std::min(1024, (9 * n_obj + 255) / 256)), 256, 0, st>>>(d_g, d_ng, n_obj, d_gss);
  h->launches += 2;
  for (int o = 0; o < n_obj && e == cudaSuccess; ++o)
    if (roms[o]->G) {
      e = launch_split_gram(roms[o]->G, roms[o]->r, roms[o]->GKK, roms[o]->GCC, roms[o]->GSk, roms[o]->gsK,
                            roms[o]->gsC, st);
      ++h->launches;
    }
  std::vector<int> flag(n_obj);
  std::vector<double> gss((size_t)n_obj * 9);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(flag.data(), d_flag, n_obj * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(gss.data(), d_gss, gss.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cleanup(MROM_ECUDA, std::string("mrom_rom_from_reduced_batch: ") + cudaGetErrorString(e));
  for (int o = 0; o < n_obj; ++o) {
    bool bad = flag[o] != 0;
    for (int k = 0; k < 9; ++k) bad = bad || !std::isfinite(roms[o]->c00[k]) || !std::isfinite(roms[o]->N0[k]);
    if (bad)
      return cleanup(MROM_EINVAL, "mrom_rom_from_reduced_batch: non-finite value in the reduced data (object " +
                                      std::to_string(o) + ")");
  }
  shared->refs = n_obj;
  for (int o = 0; o < n_obj; ++o) {
    if (roms[o]->has_cert) std::memcpy(roms[o]->gss, &gss[(size_t)o * 9], 9 * sizeof(double));
    out[o] = roms[o];
  }
  return MROM_OK;
}

extern "C" mrom_status mrom_rom_from_packed(mrom_handle h, int32_t n_obj, const mrom_packed_obj* objs,
                                            const void* packed, size_t bytes, mrom_rom_t* out) {
  if (!h) return MROM_EINVAL;
  if (n_obj < 1 || n_obj > 65535 || !objs || !packed || !out)
    return fail(h, MROM_EINVAL, "mrom_rom_from_packed: 1 <= n_obj <= 65535 and non-null arguments required");
  // region sizes and checks (host only)
  std::vector<size_t> reg(n_obj), der(n_obj);
  size_t n_der = 0;
  for (int o = 0; o < n_obj; ++o) {
    out[o] = nullptr;
    const mrom_packed_obj& d = objs[o];
    const size_t r = (size_t)d.r, rr = r * r, ng = 2 * r + 3;
    const std::string tag = " (object " + std::to_string(o) + ")";
    if (d.r < 1 || d.r > MROM_MAX_R) return fail(h, MROM_EINVAL, "mrom_rom_from_packed: r must be in [1, MROM_MAX_R]" + tag);
    if (!std::isfinite(d.alpha) || !(d.alpha > 0) || !std::isfinite(d.vol_B))
      return fail(h, MROM_EINVAL, "mrom_rom_from_packed: alpha must be finite and > 0" + tag);
    if (d.has_gram && !(d.alpha_lb > 0 && std::isfinite(d.alpha_lb)))
      return fail(h, MROM_EINVAL, "mrom_rom_from_packed: a Gram matrix needs alpha_lb > 0" + tag);
    reg[o] = (rr * (2 + (d.has_kin ? 1 : 0) + (d.has_me ? 1 : 0)) + 3 * r + (d.has_gram ? ng * ng : 0)) * 16;
    if (d.offset < 0 || d.offset % 16 != 0 || (size_t)d.offset + reg[o] > bytes)
      return fail(h, MROM_EINVAL, "mrom_rom_from_packed: region not 16-byte aligned or outside the buffer" + tag);
    bool bad = false;
    for (int k = 0; k < 9; ++k) bad = bad || !std::isfinite(d.c00[k]) || !std::isfinite(d.N0[k]);
    if (bad) return fail(h, MROM_EINVAL, "mrom_rom_from_packed: non-finite c00 or N0" + tag);
    der[o] = n_der;
    if (d.has_gram) n_der += 3 * rr + 6 * r;
  }
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  cudaStream_t st = h->stream;
  const size_t b_pack = (bytes + 255) / 256 * 256, b_der = n_der * sizeof(double2);
  const size_t b_flag = ((size_t)n_obj * sizeof(int) + 15) / 16 * 16, b_gss = (size_t)n_obj * 9 * sizeof(double);
  const size_t b_tab = (size_t)n_obj * (2 * sizeof(void*) + sizeof(size_t) + sizeof(int) + sizeof(SplitJob)) + 64;
  void* block = nullptr;
  e = cudaMallocAsync(&block, b_pack + b_der + b_flag + b_gss + b_tab, st);
  if (e != cudaSuccess) return fail(h, MROM_ENOMEM, "mrom_rom_from_packed: device allocation failed");
  char* base = static_cast<char*>(block);
  auto* derived = reinterpret_cast<double2*>(base + b_pack);
  int* d_flag = reinterpret_cast<int*>(base + b_pack + b_der);
  double* d_gss = reinterpret_cast<double*>(base + b_pack + b_der + b_flag);
  char* tab = base + b_pack + b_der + b_flag + b_gss;
  tab = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(tab) + 15) / 16 * 16);
  auto* d_jobs = reinterpret_cast<SplitJob*>(tab);
  auto** d_seg = reinterpret_cast<const double**>(tab + (size_t)n_obj * sizeof(SplitJob));
  auto** d_g = reinterpret_cast<const double2**>(d_seg + n_obj);
  auto* d_len = reinterpret_cast<size_t*>(d_g + n_obj);
  auto* d_ng = reinterpret_cast<int*>(d_len + n_obj);
  auto* shared = new mrom_rom::SharedBlock();
  shared->p = block;
  shared->stream = st;
  std::vector<mrom_rom*> roms(n_obj, nullptr);
  auto cleanup = [&](mrom_status s, const std::string& msg) {
    for (auto* m : roms) delete m;
    cudaFreeAsync(block, st);
    delete shared;
    return fail(h, s, msg);
  };
  // the whole dictionary in one copy
  e = cudaMemcpyAsync(block, packed, bytes, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_flag, 0, b_flag, st);
  std::vector<SplitJob> jobs(n_obj);
  std::vector<const double*> seg(n_obj);
  std::vector<const double2*> gp(n_obj);
  std::vector<size_t> len(n_obj);
  std::vector<int> ngv(n_obj);
  int rmax_g = 1;
  for (int o = 0; o < n_obj; ++o) {
    const mrom_packed_obj& d = objs[o];
    const size_t r = (size_t)d.r, rr = r * r, ng = 2 * r + 3;
    auto* rom = new mrom_rom();
    roms[o] = rom;
    rom->ctx = h;
    rom->r = d.r;
    rom->alpha = d.alpha;
    rom->alpha_lb = d.alpha_lb;
    rom->vol_B = d.vol_B;
    rom->shared = shared;
    auto* p = reinterpret_cast<double2*>(base + d.offset);
    rom->K = p; p += rr;
    if (d.has_kin) { rom->Kin = p; p += rr; }
    rom->C = p; p += rr;
    if (d.has_me) { rom->Me = p; p += rr; }
    rom->B = p; p += 3 * r;
    SplitJob j{};
    if (d.has_gram) {
      rom->G = p;
      double2* q = derived + der[o];
      rom->GKK = q; q += rr;
      rom->GCC = q; q += rr;
      rom->GSk = q; q += rr;
      rom->gsK = q; q += 3 * r;
      rom->gsC = q;
      j = SplitJob{rom->G, rom->GKK, rom->GCC, rom->GSk, rom->gsK, rom->gsC, d.r, 0};
      rmax_g = std::max(rmax_g, d.r);
    }
    jobs[o] = j;
    std::copy(d.c00, d.c00 + 9, rom->c00);
    std::copy(d.N0, d.N0 + 9, rom->N0);
    rom->has_cert = d.has_gram != 0;
    rom->has_kin = d.has_kin != 0;
    seg[o] = reinterpret_cast<const double*>(base + d.offset);
    len[o] = reg[o] / sizeof(double);
    gp[o] = rom->G;
    ngv[o] = (int)ng;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_jobs, jobs.data(), n_obj * sizeof(SplitJob), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_seg, seg.data(), n_obj * sizeof(void*), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_g, gp.data(), n_obj * sizeof(void*), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_len, len.data(), n_obj * sizeof(size_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_ng, ngv.data(), n_obj * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cleanup(MROM_ECUDA, std::string("mrom_rom_from_packed: upload: ") + cudaGetErrorString(e));
  nonfinite_batch_kernel<<<dim3(8, (unsigned)n_obj), 256, 0, st>>>(d_seg, d_len, d_flag);
  gather_gss_kernel<<<std::max(1, std::min(1024, (9 * n_obj + 255) / 256)), 256, 0, st>>>(d_g, d_ng, n_obj, d_gss);
  split_gram_batch_kernel<<<dim3((unsigned)std::max(1, std::min(64, (rmax_g * rmax_g + 3 * rmax_g + 255) / 256)),
                                 (unsigned)n_obj), 256, 0, st>>>(d_jobs);
  h->launches += 3;
  std::vector<int> flag(n_obj);
  std::vector<double> gss((size_t)n_obj * 9);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(flag.data(), d_flag, n_obj * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(gss.data(), d_gss, gss.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cleanup(MROM_ECUDA, std::string("mrom_rom_from_packed: ") + cudaGetErrorString(e));
  for (int o = 0; o < n_obj; ++o)
    if (flag[o])
      return cleanup(MROM_EINVAL, "mrom_rom_from_packed: non-finite value in the reduced data (object " +
                                      std::to_string(o) + ")");
  shared->refs = n_obj;
  for (int o = 0; o < n_obj; ++o) {
    if (roms[o]->has_cert) std::memcpy(roms[o]->gss, &gss[(size_t)o * 9], 9 * sizeof(double));
    out[o] = roms[o];
  }
  return MROM_OK;
}
