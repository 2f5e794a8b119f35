// Resident particle data set and its acceleration structure.
//
// Particles are grouped in h-levels (level l holds h in [h_min 2^l, h_min 2^(l+1))),
// sorted by a 48-bit Morton code of their position within each level, and cut
// into chunks of at most 32 consecutive particles that never straddle a level.
// Each chunk records its tight bounding box and its largest smoothing length,
// which is all the per-frame binning needs: a ray can only meet a particle of
// the chunk if it passes within q * h_max of the box.  Storage per particle is
// float4 (x, y, z, h) + float amplitude + int original index.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "sphdvr_internal.h"

namespace sphdvr {
namespace {

__device__ __forceinline__ unsigned f2ord(float x) {
  unsigned b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__host__ __device__ inline float ord2f(unsigned o) {
  unsigned b = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  std::memcpy(&f, &b, 4);
  return f;
#endif
}

// red[0..2] min xyz, red[3..5] max xyz, red[6] min h, red[7] max h (ordered uints); bad counts invalid rows.
__global__ void k_prep(int64_t n, const float* pos, const float* h, const float* mass, const float* dens,
                       const float* val, float* amp, unsigned* red, unsigned long long* bad) {
  unsigned mn[4] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[4] = {0, 0, 0, 0};
  unsigned long long nbad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2], hi = h[i];
    float m = mass ? mass[i] : 1.f, rho = dens ? dens[i] : 1.f, v = val ? val[i] : 1.f;
    bool ok = isfinite(x) && isfinite(y) && isfinite(z) && isfinite(hi) && hi > 0.f && isfinite(m) &&
              isfinite(rho) && rho != 0.f && isfinite(v);
    if (!ok) { ++nbad; amp[i] = 0.f; continue; }
    amp[i] = m * v / rho;
    float c[4] = {x, y, z, hi};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      unsigned o = f2ord(c[k]);
      mn[k] = min(mn[k], o);
      mx[k] = max(mx[k], o);
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      mn[k] = min(mn[k], __shfl_xor_sync(kFull, mn[k], off));
      mx[k] = max(mx[k], __shfl_xor_sync(kFull, mx[k], off));
    }
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) nbad += __shfl_xor_sync(kFull, nbad, off);
  if ((threadIdx.x & 31) == 0) {
    for (int k = 0; k < 3; ++k) { atomicMin(&red[k], mn[k]); atomicMax(&red[3 + k], mx[k]); }
    atomicMin(&red[6], mn[3]);
    atomicMax(&red[7], mx[3]);
    if (nbad) atomicAdd(bad, nbad);
  }
}

__device__ __forceinline__ uint64_t spread3(uint32_t v) {  // 16 bits -> every third bit
  uint64_t x = v & 0xffffu;
  x = (x | (x << 16)) & 0x0000ff0000ffull;
  x = (x | (x << 8)) & 0x00f00f00f00full;
  x = (x | (x << 4)) & 0x0c30c30c30c3ull;
  x = (x | (x << 2)) & 0x249249249249ull;
  return x;
}

__global__ void k_keys(int64_t n, const float* pos, const float* h, float3 lo, float3 scale, float hmin, int nlev,
                       uint64_t* keys, uint32_t* vals, unsigned* level_count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int lv = (int)floorf(log2f(h[i] / hmin));
    lv = max(0, min(nlev - 1, lv));
    uint32_t qx = (uint32_t)fminf(fmaxf((pos[3 * i] - lo.x) * scale.x, 0.f), 65535.f);
    uint32_t qy = (uint32_t)fminf(fmaxf((pos[3 * i + 1] - lo.y) * scale.y, 0.f), 65535.f);
    uint32_t qz = (uint32_t)fminf(fmaxf((pos[3 * i + 2] - lo.z) * scale.z, 0.f), 65535.f);
    keys[i] = ((uint64_t)lv << 48) | spread3(qx) | (spread3(qy) << 1) | (spread3(qz) << 2);
    vals[i] = (uint32_t)i;
    atomicAdd(&level_count[lv], 1u);
  }
}

__global__ void k_gather(int64_t n, const uint64_t* keys, const uint32_t* vals, const float* pos, const float* h,
                         const float* amp_in, const int64_t* level_start, const int64_t* level_end,
                         const int* chunk_base, float4* pos4, float* amp, int* orig, int2* chunk) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int lv = (int)(keys[i] >> 48);
    uint32_t o = vals[i];
    pos4[i] = make_float4(pos[3 * (int64_t)o], pos[3 * (int64_t)o + 1], pos[3 * (int64_t)o + 2], h[o]);
    amp[i] = amp_in[o];
    orig[i] = (int)o;
    int64_t r = i - level_start[lv];
    if ((r % kChunk) == 0) {
      int c = chunk_base[lv] + (int)(r / kChunk);
      chunk[c] = make_int2((int)i, (int)min((int64_t)kChunk, level_end[lv] - i));
    }
  }
}

__global__ void k_chunk_boxes(int n_chunks, const int2* chunk, const float4* pos4, float4* lo, float4* hi) {
  int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (c >= n_chunks) return;
  int2 ch = chunk[c];
  float4 p = pos4[ch.x + min(lane, ch.y - 1)];
  float mnx = p.x, mny = p.y, mnz = p.z, mxx = p.x, mxy = p.y, mxz = p.z, mh = p.w;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    mnx = fminf(mnx, __shfl_xor_sync(kFull, mnx, o));
    mny = fminf(mny, __shfl_xor_sync(kFull, mny, o));
    mnz = fminf(mnz, __shfl_xor_sync(kFull, mnz, o));
    mxx = fmaxf(mxx, __shfl_xor_sync(kFull, mxx, o));
    mxy = fmaxf(mxy, __shfl_xor_sync(kFull, mxy, o));
    mxz = fmaxf(mxz, __shfl_xor_sync(kFull, mxz, o));
    mh = fmaxf(mh, __shfl_xor_sync(kFull, mh, o));
  }
  if (lane == 0) {
    lo[c] = make_float4(mnx, mny, mnz, mh);
    hi[c] = make_float4(mxx, mxy, mxz, (float)ch.y);
  }
}

}  // namespace

sphdvr_status build_dataset(sphdvr_ctx* ctx, sphdvr_dataset* ds, const float* pos, const float* h,
                            const float* mass, const float* density, const float* value, cudaStream_t st) {
  const int64_t n = ds->n;
  sphdvr_status s;
  cudaError_t e;
  float* amp_tmp = nullptr;
  unsigned* red = nullptr;
  unsigned long long* bad = nullptr;
  uint64_t *keys = nullptr, *keys2 = nullptr;
  uint32_t *vals = nullptr, *vals2 = nullptr;
  unsigned* lcount = nullptr;
  int64_t* lbounds = nullptr;
  int* cbase = nullptr;
  auto cleanup = [&]() {
    cudaFree(amp_tmp); cudaFree(red); cudaFree(bad); cudaFree(keys); cudaFree(keys2); cudaFree(vals);
    cudaFree(vals2); cudaFree(lcount); cudaFree(lbounds); cudaFree(cbase);
  };
  if ((s = dev_alloc(ctx, (void**)&amp_tmp, n * sizeof(float))) != SPHDVR_OK ||
      (s = dev_alloc(ctx, (void**)&red, 8 * sizeof(unsigned))) != SPHDVR_OK ||
      (s = dev_alloc(ctx, (void**)&bad, sizeof(unsigned long long))) != SPHDVR_OK) {
    cleanup();
    return s;
  }
  unsigned init[8] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0, 0, 0, 0xffffffffu, 0};
  cudaMemcpyAsync(red, init, sizeof(init), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(bad, 0, sizeof(unsigned long long), st);
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
  k_prep<<<blocks, 256, 0, st>>>(n, pos, h, mass, density, value, amp_tmp, red, bad);
  ++ctx->launches;
  unsigned hred[8];
  unsigned long long hbad = 0;
  cudaMemcpyAsync(hred, red, sizeof(hred), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, st);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { cleanup(); return cuda_err(ctx, e, "dataset prep"); }
  if (hbad) {
    cleanup();
    return set_err(ctx, SPHDVR_EINVAL, "dataset: " + std::to_string(hbad) + " particles with non-finite data, h <= 0 or density 0");
  }
  float lo[3], hi[3];
  for (int k = 0; k < 3; ++k) { lo[k] = ord2f(hred[k]); hi[k] = ord2f(hred[3 + k]); }
  float hmin = ord2f(hred[6]), hmax = ord2f(hred[7]);
  int nlev = std::max(1, std::min(40, (int)std::floor(std::log2((double)hmax / hmin)) + 1));
  float3 lo3 = make_float3(lo[0], lo[1], lo[2]);
  float3 sc;
  sc.x = 65535.f / std::max(hi[0] - lo[0], 1e-30f);
  sc.y = 65535.f / std::max(hi[1] - lo[1], 1e-30f);
  sc.z = 65535.f / std::max(hi[2] - lo[2], 1e-30f);
  if ((s = dev_alloc(ctx, (void**)&keys, n * 8)) != SPHDVR_OK || (s = dev_alloc(ctx, (void**)&keys2, n * 8)) != SPHDVR_OK ||
      (s = dev_alloc(ctx, (void**)&vals, n * 4)) != SPHDVR_OK || (s = dev_alloc(ctx, (void**)&vals2, n * 4)) != SPHDVR_OK ||
      (s = dev_alloc(ctx, (void**)&lcount, 64 * sizeof(unsigned))) != SPHDVR_OK) {
    cleanup();
    return s;
  }
  cudaMemsetAsync(lcount, 0, 64 * sizeof(unsigned), st);
  k_keys<<<blocks, 256, 0, st>>>(n, pos, h, lo3, sc, hmin, nlev, keys, vals, lcount);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) { cleanup(); return cuda_err(ctx, e, "k_keys"); }
  int lbits = 0;
  while ((1 << lbits) < nlev) ++lbits;
  if ((s = ensure(ctx, ctx->sort_tmp, sort_tmp_words(n) * sizeof(uint32_t))) != SPHDVR_OK) { cleanup(); return s; }
  s = radix_sort_u64(ctx, keys, vals, keys2, vals2, n, 48 + lbits, (uint32_t*)ctx->sort_tmp.p, st);
  if (s != SPHDVR_OK) { cleanup(); return s; }
  unsigned hcount[64];
  cudaMemcpyAsync(hcount, lcount, sizeof(hcount), cudaMemcpyDeviceToHost, st);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { cleanup(); return cuda_err(ctx, e, "dataset sort"); }
  std::vector<int64_t> hb(2 * 64, 0);
  std::vector<int> hbase(64, 0);
  int64_t acc = 0;
  int nch = 0;
  for (int l = 0; l < nlev; ++l) {
    hb[l] = acc;
    acc += hcount[l];
    hb[64 + l] = acc;
    hbase[l] = nch;
    nch += (int)((hcount[l] + kChunk - 1) / kChunk);
  }
  if ((s = dev_alloc(ctx, (void**)&lbounds, 2 * 64 * sizeof(int64_t))) != SPHDVR_OK ||
      (s = dev_alloc(ctx, (void**)&cbase, 64 * sizeof(int))) != SPHDVR_OK) {
    cleanup();
    return s;
  }
  cudaMemcpyAsync(lbounds, hb.data(), 2 * 64 * sizeof(int64_t), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(cbase, hbase.data(), 64 * sizeof(int), cudaMemcpyHostToDevice, st);
  ds->n_levels = nlev;
  ds->n_chunks = nch;
  if ((s = dev_alloc(ctx, (void**)&ds->pos, n * sizeof(float4))) != SPHDVR_OK ||
      (s = dev_alloc(ctx, (void**)&ds->amp, n * sizeof(float))) != SPHDVR_OK ||
      (s = dev_alloc(ctx, (void**)&ds->orig, n * sizeof(int))) != SPHDVR_OK ||
      (s = dev_alloc(ctx, (void**)&ds->chunk, nch * sizeof(int2))) != SPHDVR_OK ||
      (s = dev_alloc(ctx, (void**)&ds->chunk_lo, nch * sizeof(float4))) != SPHDVR_OK ||
      (s = dev_alloc(ctx, (void**)&ds->chunk_hi, nch * sizeof(float4))) != SPHDVR_OK) {
    cleanup();
    return s;
  }
  ds->bytes = n * (sizeof(float4) + sizeof(float) + sizeof(int)) + nch * (sizeof(int2) + 2 * sizeof(float4));
  k_gather<<<blocks, 256, 0, st>>>(n, keys, vals, pos, h, amp_tmp, lbounds, lbounds + 64, cbase, ds->pos, ds->amp,
                                   ds->orig, ds->chunk);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) { cleanup(); return cuda_err(ctx, e, "k_gather"); }
  k_chunk_boxes<<<(nch + 7) / 8, 256, 0, st>>>(nch, ds->chunk, ds->pos, ds->chunk_lo, ds->chunk_hi);
  ++ctx->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) { cleanup(); return cuda_err(ctx, e, "k_chunk_boxes"); }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { cleanup(); return cuda_err(ctx, e, "dataset build"); }
  cleanup();
  return SPHDVR_OK;
}

}  // namespace sphdvr
