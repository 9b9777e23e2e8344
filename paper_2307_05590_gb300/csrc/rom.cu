// Reduced objects: device storage, input checks and the certificate Gram split.
#include "mrom_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>

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

extern "C" void mrom_rom_free(mrom_rom_t rom) {
  if (!rom) return;
  if (rom->d_block) cudaFree(rom->d_block);
  delete rom;
}
