// Quantum values of a resident data set (Sec. 4.4): sigma = A_max / int_max with
// A_max an upper bound of the field, tau minimising the quantisation error
// estimate of a representative particle.  The paper leaves the bound to "a
// short analysis of the data set"; here it is rigorous: every particle's peak
// value c w(0) (c = m v / (rho h^3)) is added to each cell of a uniform grid
// over the data set's bounding box (cells about the representative support
// radius, at most kGrid per axis) that its support meets -- at any point the
// field is a sum of contributions no larger than their peaks from particles
// whose supports contain the point, hence meet the point's cell -- and A_max
// is the largest cell sum (of absolute peaks), with a 1 % margin for the
// piecewise approximation and FP32 sums.  A particle whose support meets more than
// kMaxCells cells adds its peak to every cell at once (a common offset).  The
// representative particle has the median smoothing length and the median c
// (upper medians: element n / 2 in order).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "device_common.cuh"
#include "sphdvr_internal.h"

namespace sphdvr {
namespace {

constexpr int kGrid = 128;        // cells per axis
constexpr int kMaxCells = 4096;   // larger supports go to the common offset

__global__ void k_peak_deposit(int64_t n, const float4* pos, const float* amp, float w0, float q, float3 lo,
                               float inv_cs, int3 dim, float* cells, float* offset) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 P = pos[i];
  const float peak = fabsf(amp[i]) / (P.w * P.w * P.w) * w0, R = q * P.w;
  int c0[3], c1[3];
  const float x[3] = {P.x, P.y, P.z}, l[3] = {lo.x, lo.y, lo.z};
  const int g[3] = {dim.x, dim.y, dim.z};
  long long cnt = 1;
  for (int a = 0; a < 3; ++a) {
    c0[a] = max(0, min(g[a] - 1, (int)floorf((x[a] - R - l[a]) * inv_cs)));
    c1[a] = max(0, min(g[a] - 1, (int)floorf((x[a] + R - l[a]) * inv_cs)));
    cnt *= c1[a] - c0[a] + 1;
  }
  if (cnt > kMaxCells) {
    atomicAdd(offset, peak);
    return;
  }
  for (int z = c0[2]; z <= c1[2]; ++z)
    for (int y = c0[1]; y <= c1[1]; ++y)
      for (int xx = c0[0]; xx <= c1[0]; ++xx) atomicAdd(cells + ((size_t)z * g[1] + y) * g[0] + xx, peak);
}

__global__ void k_max_cells(const float* cells, int64_t n, unsigned* out) {
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, cells[i]);
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // non-negative floats order as integers
}

double median(std::vector<double>& v) {
  const size_t k = v.size() / 2;
  std::nth_element(v.begin(), v.begin() + k, v.end());
  return v[k];
}

}  // namespace
}  // namespace sphdvr

using namespace sphdvr;

extern "C" sphdvr_status sphdvr_dataset_quant_params(sphdvr_ctx* ctx, const sphdvr_dataset* ds, int kernel, int D,
                                                     int int_bits, double* tau, double* sigma, double* qe,
                                                     double* a_max) {
  if (!ctx) return SPHDVR_EINVAL;
  if (!ds || ds->ctx != ctx || !tau || !sigma || !qe || !a_max || kernel < 0 || kernel > 3 || D < 1 || D > 6 ||
      int_bits < 8 || int_bits > 1024)
    return set_err(ctx, SPHDVR_EINVAL, "dataset_quant_params: bad arguments");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  const int64_t n = ds->n;
  if (n < 1) return set_err(ctx, SPHDVR_EINVAL, "dataset_quant_params: empty data set");
  // representative particle: medians of h and of c = amp / h^3
  std::vector<float4> pos((size_t)n);
  std::vector<float> amp((size_t)n);
  std::vector<float4> clo((size_t)ds->n_chunks), chi((size_t)ds->n_chunks);
  if ((e = cudaMemcpy(pos.data(), ds->pos, (size_t)n * sizeof(float4), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(amp.data(), ds->amp, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(clo.data(), ds->chunk_lo, clo.size() * sizeof(float4), cudaMemcpyDeviceToHost)) !=
          cudaSuccess ||
      (e = cudaMemcpy(chi.data(), ds->chunk_hi, chi.size() * sizeof(float4), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_err(ctx, e, "dataset_quant_params copy");
  std::vector<double> hv((size_t)n), cv((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    const double h = pos[i].w;
    hv[i] = h;
    cv[i] = (double)amp[i] / (h * h * h);
  }
  const double h_rep = median(hv), pc_rep = median(cv);
  // bounding box of the particles' supports
  const float q = kernel == 3 ? 1.f : 2.f;
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (size_t c = 0; c < clo.size(); ++c) {
    const float r = q * clo[c].w;  // w: the chunk's largest h
    const float l[3] = {clo[c].x, clo[c].y, clo[c].z}, u[3] = {chi[c].x, chi[c].y, chi[c].z};
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], l[a] - r);
      hi[a] = std::max(hi[a], u[a] + r);
    }
  }
  // cells about as large as the representative particle's support radius, at
  // most kGrid per axis
  const float ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-30f});
  const float cs = std::max(ext / kGrid, q * (float)h_rep) * (1.f + 1e-6f);
  int3 dim;
  int* dp[3] = {&dim.x, &dim.y, &dim.z};
  for (int a = 0; a < 3; ++a) *dp[a] = std::max(1, std::min(kGrid, (int)std::ceil((hi[a] - lo[a]) / cs)));
  const size_t ncell = (size_t)dim.x * dim.y * dim.z;
  float* cells = nullptr;
  sphdvr_status s = dev_alloc(ctx, (void**)&cells, ncell * sizeof(float) + 16);
  if (s != SPHDVR_OK) return s;
  float* offset = cells + ncell;
  unsigned* mx = (unsigned*)(cells + ncell + 1);
  const float w0 = (float)kernel_peak_host(kernel);
  if ((e = cudaMemset(cells, 0, ncell * sizeof(float) + 16)) == cudaSuccess) {
    k_peak_deposit<<<(unsigned)((n + 255) / 256), 256>>>(n, ds->pos, ds->amp, w0, q, make_float3(lo[0], lo[1], lo[2]),
                                                         1.f / cs, dim, cells, offset);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_max_cells<<<1024, 256>>>(cells, (int64_t)ncell, mx);
    e = cudaGetLastError();
  }
  float host[2] = {0.f, 0.f};
  unsigned mbits = 0;
  if (e == cudaSuccess) e = cudaMemcpy(host, offset, sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&mbits, mx, sizeof(unsigned), cudaMemcpyDeviceToHost);
  cudaFree(cells);
  if (e != cudaSuccess) return cuda_err(ctx, e, "dataset_quant_params");
  float mcell;
  std::memcpy(&mcell, &mbits, sizeof(float));
  // margin: the FP32 cell sums' rounding, and the piecewise approximation of a
  // particle, which may exceed its peak by its approximation error
  const double amax = ((double)mcell + (double)host[0]) * 1.01;
  if (!(amax > 0) || !(pc_rep > 0) || !(h_rep > 0))
    return set_err(ctx, SPHDVR_EINVAL, "dataset_quant_params: field bound or representative particle is zero");
  double t_rel, s_rel, q_e;
  if (quant_params_host(kernel, D, int_bits, amax / (kernel_peak_host(kernel) * pc_rep), &t_rel, &s_rel, &q_e) != 0)
    return set_err(ctx, SPHDVR_EINVAL, "dataset_quant_params: no quantum values");
  *tau = t_rel * h_rep;
  *sigma = s_rel * pc_rep;
  *qe = q_e;
  *a_max = amax;
  return SPHDVR_OK;
}
