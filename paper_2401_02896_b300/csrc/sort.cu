// Device prefix sum and stable LSD radix sort (8-bit digits), used by the
// data-set build (Morton keys) and by the per-frame chunk-to-tile binning.
#include "device_common.cuh"
#include "sphdvr_internal.h"

namespace sphdvr {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp, uint32_t& excl) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
    uint32_t s = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(kFull, s, o);
      if (lane >= o) s += y;
    }
    if (lane < (int)(blockDim.x >> 5)) s_warp[lane] = s - t;
    if (lane == 31) s_warp[32] = s;
  }
  __syncthreads();
  excl = x - v + s_warp[w];
  uint32_t total = s_warp[32];
  __syncthreads();
  return total;
}

__global__ void k_scan_tiles(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tile_sums) {
  __shared__ uint32_t s_warp[33];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems], sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0u;
    sum += v[i];
  }
  uint32_t excl;
  uint32_t total = block_exclusive_scan(sum, s_warp, excl);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = excl;
    excl += v[i];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_add(uint32_t* out, int64_t n, const uint32_t* tile_offs) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t add = tile_offs[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) out[base + i] += add;
}

__global__ void k_scan_single(uint32_t* data, int n, uint32_t* total) {
  // exclusive scan of n <= kScanTile values in one block
  __shared__ uint32_t s_warp[33];
  int base = threadIdx.x * kScanItems;
  uint32_t v[kScanItems], sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? data[base + i] : 0u;
    sum += v[i];
  }
  uint32_t excl;
  uint32_t tot = block_exclusive_scan(sum, s_warp, excl);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) data[base + i] = excl;
    excl += v[i];
  }
  if (threadIdx.x == 0 && total) *total = tot;
}

// ---- radix sort ------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048 keys per tile
constexpr int kWarps = kSortThreads / 32;

__global__ void k_radix_hist(const uint64_t* keys, int64_t n, int shift, uint32_t* hist, int n_tiles) {
  __shared__ uint32_t s_h[256];
  s_h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    int64_t idx = base + i * kSortThreads + threadIdx.x;
    if (idx < n) atomicAdd(&s_h[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = s_h[threadIdx.x];
}

// Stable scatter: keys are taken in rounds of kSortThreads (round-major, then
// thread order), which is their original order within the tile.
__global__ void k_radix_scatter(const uint64_t* keys, const uint32_t* vals, uint64_t* okeys, uint32_t* ovals,
                                int64_t n, int shift, const uint32_t* offs, int n_tiles) {
  __shared__ uint32_t s_cnt[kWarps][256];
  __shared__ uint32_t s_run[256];
  __shared__ uint32_t s_base[256];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  s_run[threadIdx.x] = 0;
  s_base[threadIdx.x] = offs[(int64_t)threadIdx.x * n_tiles + blockIdx.x];
  int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortItems; ++r) {
    for (int i = threadIdx.x; i < kWarps * 256; i += kSortThreads) (&s_cnt[0][0])[i] = 0;
    __syncthreads();
    int64_t idx = base + r * kSortThreads + threadIdx.x;
    bool ok = idx < n;
    uint64_t k = ok ? keys[idx] : 0;
    uint32_t v = ok ? vals[idx] : 0;
    uint32_t d = ok ? (uint32_t)((k >> shift) & 255u) : 256u + lane;  // invalid lanes get unique groups
    unsigned peers = __match_any_sync(kFull, d);
    int rank = __popc(peers & lanemask_lt());
    if (ok && rank == 0) s_cnt[w][d] = __popc(peers);
    __syncthreads();
    {  // per digit: exclusive offsets over warps, running count over rounds
      int dd = threadIdx.x;
      uint32_t run = s_run[dd];
      for (int ww = 0; ww < kWarps; ++ww) {
        uint32_t c = s_cnt[ww][dd];
        s_cnt[ww][dd] = run;
        run += c;
      }
      s_run[dd] = run;
    }
    __syncthreads();
    if (ok) {
      uint32_t pos = s_base[d] + s_cnt[w][d] + rank;
      okeys[pos] = k;
      ovals[pos] = v;
    }
    __syncthreads();
  }
}

}  // namespace

size_t scan_tmp_words(int64_t n) {
  size_t need = 16;
  for (int64_t t = (n + kScanTile - 1) / kScanTile; t > 1; t = (t + kScanTile - 1) / kScanTile) need += (size_t)t + 1;
  return need;
}

size_t sort_tmp_words(int64_t n) {
  int64_t tiles = (n + kSortTile - 1) / kSortTile;
  size_t hist_n = (size_t)tiles * 256;
  return hist_n + scan_tmp_words((int64_t)hist_n);
}

sphdvr_status scan_exclusive_u32(sphdvr_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total,
                                 uint32_t* tmp, cudaStream_t st) {
  if (n <= 0) {
    if (total) {
      cudaError_t e = cudaMemsetAsync(total, 0, sizeof(uint32_t), st);
      if (e != cudaSuccess) return cuda_err(ctx, e, "scan memset");
    }
    return SPHDVR_OK;
  }
  if (n <= kScanTile) {
    if (in != out) {
      cudaError_t e = cudaMemcpyAsync(out, in, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return cuda_err(ctx, e, "scan copy");
    }
    k_scan_single<<<1, kScanThreads, 0, st>>>(out, (int)n, total);
    ++ctx->launches;
    return cuda_err(ctx, cudaGetLastError(), "k_scan_single");
  }
  // reduce-then-scan: tile sums of each level placed consecutively in tmp
  std::vector<std::pair<uint32_t*, int64_t>> levels;
  uint32_t* cur_out = out;
  const uint32_t* cur_in = in;
  int64_t cur_n = n;
  size_t used = 0;
  while (cur_n > kScanTile) {
    int64_t t = (cur_n + kScanTile - 1) / kScanTile;
    uint32_t* sums = tmp + used;
    used += (size_t)t + 1;
    k_scan_tiles<<<(unsigned)t, kScanThreads, 0, st>>>(cur_in, cur_out, cur_n, sums);
    ++ctx->launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(ctx, e, "k_scan_tiles");
    levels.push_back({cur_out, cur_n});
    cur_in = sums;
    cur_out = sums;
    cur_n = t;
  }
  k_scan_single<<<1, kScanThreads, 0, st>>>(cur_out, (int)cur_n, total);
  ++ctx->launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "k_scan_single");
  // propagate the scanned sums of level i (stored where level i+1 was scanned in place) down
  for (int i = (int)levels.size() - 1; i >= 0; --i) {
    int64_t t = (levels[i].second + kScanTile - 1) / kScanTile;
    const uint32_t* offs = (i == (int)levels.size() - 1) ? cur_out : levels[i + 1].first;
    k_scan_add<<<(unsigned)t, kScanThreads, 0, st>>>(levels[i].first, levels[i].second, offs);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(ctx, e, "k_scan_add");
  }
  return SPHDVR_OK;
}

sphdvr_status radix_sort_u64(sphdvr_ctx* ctx, uint64_t* keys, uint32_t* vals, uint64_t* keys2, uint32_t* vals2,
                             int64_t n, int nbits, uint32_t* tmp, cudaStream_t st) {
  if (n <= 1) return SPHDVR_OK;
  int64_t tiles = (n + kSortTile - 1) / kSortTile;
  size_t hist_n = (size_t)tiles * 256;
  uint32_t* hist = tmp;
  uint32_t* scan_tmp = tmp + hist_n;
  int passes = (nbits + 7) / 8;
  uint64_t *ka = keys, *kb = keys2;
  uint32_t *va = vals, *vb = vals2;
  for (int p = 0; p < passes; ++p) {
    int shift = 8 * p;
    k_radix_hist<<<(unsigned)tiles, kSortThreads, 0, st>>>(ka, n, shift, hist, (int)tiles);
    ++ctx->launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(ctx, e, "k_radix_hist");
    sphdvr_status s = scan_exclusive_u32(ctx, hist, hist, (int64_t)hist_n, nullptr, scan_tmp, st);
    if (s != SPHDVR_OK) return s;
    k_radix_scatter<<<(unsigned)tiles, kSortThreads, 0, st>>>(ka, va, kb, vb, n, shift, hist, (int)tiles);
    ++ctx->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(ctx, e, "k_radix_scatter");
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    cudaError_t e = cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_err(ctx, e, "radix copy back");
  }
  return SPHDVR_OK;
}

}  // namespace sphdvr
