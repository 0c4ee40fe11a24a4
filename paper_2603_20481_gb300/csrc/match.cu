// Detection quality on the GPU (Sec. III-A-2, Eqs. 2 and 3): for every
// ground-truth box its best IoU over the detections, for every detection its
// best IoU over the ground truth (the row and column maxima of the IoU
// matrix, which is never stored), and N_t, N_f at any number of IoU
// thresholds.  The best IoU of a box is kept exactly, as its (intersection,
// union) pair: fractions are compared by 128-bit cross products.
#include <algorithm>
#include <cstring>
#include <vector>

#include "context.cuh"

namespace rise {
namespace {

constexpr int MT_THREADS = 256;
constexpr int MT_TILE = 2048;   // boxes of the other set staged per block step (32 KB)

__device__ __forceinline__ int64_t cells(int4 b) {
  return ((int64_t)b.y - b.x + 1) * ((int64_t)b.w - b.z + 1);
}

// best[i] = (intersection, union) of box i of A with its best box of B.
__global__ void __launch_bounds__(MT_THREADS)
best_iou_kernel(const int4 *A, int64_t na, const int4 *B, int64_t nb, ulonglong2 *best) {
  __shared__ int4 tile[MT_TILE];
  for (int64_t i0 = (int64_t)blockIdx.x * MT_THREADS; i0 < na; i0 += (int64_t)gridDim.x * MT_THREADS) {
    const int64_t i = i0 + threadIdx.x;
    const bool live = i < na;
    const int4 a = live ? A[i] : make_int4(0, 0, 0, 0);
    const int64_t aa = cells(a);
    uint64_t bi = 0, bu = 1;
    for (int64_t j0 = 0; j0 < nb; j0 += MT_TILE) {
      const int nt = (int)min((int64_t)MT_TILE, nb - j0);
      __syncthreads();
      for (int k = threadIdx.x; k < nt; k += MT_THREADS) tile[k] = B[j0 + k];
      __syncthreads();
      if (live) {
        for (int k = 0; k < nt; ++k) {
          const int4 b = tile[k];
          const int64_t t = (int64_t)min(a.y, b.y) - max(a.x, b.x) + 1;
          const int64_t f = (int64_t)min(a.w, b.w) - max(a.z, b.z) + 1;
          if (t <= 0 || f <= 0) continue;
          const uint64_t in = (uint64_t)(t * f);
          const uint64_t un = (uint64_t)(aa + cells(b)) - in;
          if ((unsigned __int128)in * bu > (unsigned __int128)bi * un) {
            bi = in;
            bu = un;
          }
        }
      }
    }
    if (live) best[i] = make_ulonglong2(bi, bu);
  }
}

// counts[2k] += boxes of the ground truth with best IoU > theta[k],
// counts[2k+1] += detections with best IoU < theta[k]  (Eq. 2)
__global__ void iou_count_kernel(const ulonglong2 *gbest, int64_t ng, const ulonglong2 *dbest,
                                 int64_t nd, const double *theta, int nth,
                                 unsigned long long *counts) {
  const int k = blockIdx.y;
  const double th = theta[k];
  unsigned long long t = 0, f = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ng + nd;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < ng) {
      const ulonglong2 b = gbest[i];
      t += (double)b.x > __dmul_rn(th, (double)b.y);
    } else {
      const ulonglong2 b = dbest[i - ng];
      f += (double)b.x < __dmul_rn(th, (double)b.y);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    t += __shfl_xor_sync(0xffffffffu, t, o);
    f += __shfl_xor_sync(0xffffffffu, f, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (t) atomicAdd(&counts[2 * k], t);
    if (f) atomicAdd(&counts[2 * k + 1], f);
  }
}

}  // namespace

void match_preload() {
  preload_kernel(best_iou_kernel);
  preload_kernel(iou_count_kernel);
}
}  // namespace rise

using namespace rise;
using namespace rise::host;

extern "C" int rise_match_boxes(rise_ctx *c, const int32_t *gt, int64_t n_gt, const rise_box *det,
                                int64_t n_det, const double *thetas, int n_theta, int64_t *n_t,
                                int64_t *n_f, int64_t *gt_best, int64_t *det_best) {
  if (!c || n_gt < 0 || n_det < 0 || n_theta < 0 || n_theta > 65535) return RISE_EINVAL;
  if ((n_gt && !gt) || (n_det && !det) || (n_theta && (!thetas || !n_t || !n_f))) return RISE_EINVAL;
  if (c->npend) return RISE_EINVAL;
  for (int64_t i = 0; i < n_gt; ++i)
    if (gt[4 * i + 1] < gt[4 * i] || gt[4 * i + 3] < gt[4 * i + 2]) return RISE_EINVAL;
  for (int k = 0; k < n_theta; ++k)
    if (!(thetas[k] >= 0.0 && thetas[k] <= 1.0)) return RISE_EINVAL;
  CK(cudaSetDevice(c->device));
  // boxes as int4 (t0, t1, f0, f1), ground truth first, then detections
  const int64_t nall = n_gt + n_det;
  std::vector<int4> boxes((size_t)std::max<int64_t>(nall, 1));
  for (int64_t i = 0; i < n_gt; ++i)
    boxes[i] = make_int4(gt[4 * i], gt[4 * i + 1], gt[4 * i + 2], gt[4 * i + 3]);
  for (int64_t j = 0; j < n_det; ++j)
    boxes[n_gt + j] = make_int4(det[j].t0, det[j].t1, det[j].f0, det[j].f1);
  int rc;
  const size_t nb_box = sizeof(int4) * (size_t)std::max<int64_t>(nall, 1);
  const size_t nb_best = sizeof(ulonglong2) * (size_t)std::max<int64_t>(nall, 1);
  if ((rc = ensure(c, c->match_boxes, nb_box))) return rc;
  if ((rc = ensure(c, c->match_best, nb_best))) return rc;
  if ((rc = ensure(c, c->match_misc, sizeof(double) * 65536 + 2 * sizeof(uint64_t) * 65536))) return rc;
  cudaStream_t s = c->stream;
  int4 *dbox = static_cast<int4 *>(c->match_boxes.p);
  ulonglong2 *dbest = static_cast<ulonglong2 *>(c->match_best.p);
  double *dth = static_cast<double *>(c->match_misc.p);
  unsigned long long *dcnt = reinterpret_cast<unsigned long long *>(dth + 65536);
  if (nall) CK(cudaMemcpyAsync(dbox, boxes.data(), sizeof(int4) * nall, cudaMemcpyHostToDevice, s));
  if (n_theta) {
    CK(cudaMemcpyAsync(dth, thetas, sizeof(double) * n_theta, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(dcnt, 0, 2 * sizeof(uint64_t) * n_theta, s));
  }
  const int cap_blocks = c->num_sms * 8;
  if (n_gt) {
    const int g = (int)std::min<int64_t>((n_gt + MT_THREADS - 1) / MT_THREADS, cap_blocks);
    best_iou_kernel<<<g, MT_THREADS, 0, s>>>(dbox, n_gt, dbox + n_gt, n_det, dbest);
    count_launches(1);
  }
  if (n_det) {
    const int g = (int)std::min<int64_t>((n_det + MT_THREADS - 1) / MT_THREADS, cap_blocks);
    best_iou_kernel<<<g, MT_THREADS, 0, s>>>(dbox + n_gt, n_det, dbox, n_gt, dbest + n_gt);
    count_launches(1);
  }
  if (n_theta && nall) {
    const int g = (int)std::min<int64_t>((nall + 255) / 256, 64);
    iou_count_kernel<<<dim3(g, n_theta), 256, 0, s>>>(dbest, n_gt, dbest + n_gt, n_det, dth, n_theta, dcnt);
    count_launches(1);
  }
  CK(cudaGetLastError());
  std::vector<uint64_t> cnt(2 * (size_t)std::max(n_theta, 1), 0);
  if (n_theta) CK(cudaMemcpyAsync(cnt.data(), dcnt, 2 * sizeof(uint64_t) * n_theta, cudaMemcpyDeviceToHost, s));
  if (gt_best && n_gt) CK(cudaMemcpyAsync(gt_best, dbest, sizeof(ulonglong2) * n_gt, cudaMemcpyDeviceToHost, s));
  if (det_best && n_det)
    CK(cudaMemcpyAsync(det_best, dbest + n_gt, sizeof(ulonglong2) * n_det, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int k = 0; k < n_theta; ++k) {
    n_t[k] = (int64_t)cnt[2 * k];
    n_f[k] = (int64_t)cnt[2 * k + 1];
  }
  return RISE_OK;
}
