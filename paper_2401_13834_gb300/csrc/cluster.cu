// Candidate clustering on the GPU (Sec. 2.5): DBSCAN on the DM-time plane,
// with DM converted to dispersion delay across the band (Eq. 1) so that both
// axes are in milliseconds.
//
//   core point      more than k other points at distance <= r
//   cluster         the core points connected by chains of core neighbours,
//                   with the non-core points within r of them
//   outlier         any other point
//
// The paper finds neighbours with a kd-tree (Sec. 2.5, O(log N) per query);
// on the GPU a uniform grid of cells slightly larger than r does the same
// job: every neighbour of a point lies in the 3 x 3 cells around it, and the
// points sorted by cell make each cell row one contiguous range.
//
// Steps (one stream, no host round trip):
//   1. canonical order: points sorted by (DM index, time) (radix sort);
//   2. coordinates (delay table, t * t_samp) and cell keys; points sorted by cell;
//   3. neighbour counts -> core flags;
//   4. union-find over core pairs (lock-free: a root is linked under a smaller
//      root, so the final root of a cluster is its smallest canonical index,
//      which is the cluster's id);
//   5. labels: a core point's root; a non-core point the smallest root among
//      its core neighbours, or -1;
//   6. per cluster: member count, DM and time extent, and the member of
//      highest S/N (ties: smallest canonical index), by integer atomics;
//   7. compaction of the clusters in id order (exclusive scan).
// Every result is independent of thread order.
#include <cuda_runtime.h>

#include <cub/cub.cuh>

#include <algorithm>
#include <cstring>
#include <new>

#include "tx_internal.h"

using namespace tx;

#define TX_CUDA(expr)                                                               \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      set_error("%s failed: %s", #expr, cudaGetErrorString(e_));                    \
      return TX_ERR_CUDA;                                                           \
    }                                                                               \
  } while (0)

struct tx_clusterer {
  int device = -1;
  double r = 0.0, cell = 0.0, tsamp_ms = 0.0;
  int32_t k = 0;
  int64_t cap = 0;
  int ndm = 0;
  double* table = nullptr;              // [ndm] delay per DM trial, ms
  unsigned long long *key_a = nullptr, *key_b = nullptr;
  int32_t *val_a = nullptr, *val_b = nullptr;
  int32_t* perm = nullptr;              // canonical index -> record index
  double *x = nullptr, *y = nullptr;    // canonical coordinates
  unsigned long long* ckey = nullptr;   // cell keys sorted
  int32_t* cidx = nullptr;              // canonical index of each sorted cell entry
  float *xs = nullptr, *ys = nullptr;   // per sorted entry: coordinates relative to its cell corner
  int32_t* core = nullptr;
  int32_t* parent = nullptr;
  int32_t* label = nullptr;
  int32_t* cnt = nullptr;
  unsigned long long* rep = nullptr;
  int32_t *dlo = nullptr, *dhi = nullptr, *tlo = nullptr, *thi = nullptr;
  int32_t* flag = nullptr;
  int32_t* pos = nullptr;
  void* temp = nullptr;
  size_t temp_bytes = 0;
};

namespace {

constexpr int kThreads = 256;

__global__ void k_cl_canon(const tx_cand* __restrict__ c, int n, unsigned long long* key, int32_t* val) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  key[i] = ((unsigned long long)(uint32_t)c[i].dm_index << 32) | (uint32_t)c[i].t;
  val[i] = i;
}

__global__ void k_cl_coords(const tx_cand* __restrict__ c, const int32_t* __restrict__ perm, int n,
                            const double* __restrict__ table, double tsamp_ms, double cell, double* x, double* y,
                            unsigned long long* key, int32_t* val) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const tx_cand r = c[perm[j]];
  const double xv = table[r.dm_index];
  const double yv = __dmul_rn((double)r.t, tsamp_ms);
  x[j] = xv;
  y[j] = yv;
  const unsigned long long cx = (unsigned long long)floor(xv / cell), cy = (unsigned long long)floor(yv / cell);
  key[j] = (cx << 32) | cy;
  val[j] = j;
}

__device__ __forceinline__ int lower_bound(const unsigned long long* __restrict__ a, int n, unsigned long long v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Calls f(q) for every other point q within r of canonical point j, in cell
// order; f returns false to stop early. The test is
//   (x_q - x_j)^2 + (y_q - y_j)^2 <= r^2     in IEEE double,
// screened first in float on coordinates relative to the cell corner (errors
// below 1e-6 r^2): only pairs within 1e-5 r^2 of the radius take the double
// test, so every decision is the double one.
template <typename F>
__device__ __forceinline__ void for_neighbours(const tx_clusterer& C, int n, int j, F&& f) {
  const double xj = C.x[j], yj = C.y[j];
  const double r2 = __dmul_rn(C.r, C.r);
  const float r2f = (float)r2, lo2 = r2f * (1.0f - 1e-5f), hi2 = r2f * (1.0f + 1e-5f);
  const float cellf = (float)C.cell;
  const long long cx = (long long)floor(xj / C.cell), cy = (long long)floor(yj / C.cell);
  const float xjl = (float)(xj - (double)cx * C.cell), yjl = (float)(yj - (double)cy * C.cell);
  for (long long dx = -1; dx <= 1; ++dx) {
    if (cx + dx < 0) continue;
    const unsigned long long row = (unsigned long long)(cx + dx) << 32;
    const unsigned long long lo = row | (unsigned long long)(cy > 0 ? cy - 1 : 0);
    const unsigned long long hi = row | (unsigned long long)(cy + 1);
    for (int e = lower_bound(C.ckey, n, lo); e < n; ++e) {
      const unsigned long long key = C.ckey[e];
      if (key > hi) break;
      const float ddx = C.xs[e] - xjl + (float)dx * cellf;
      const float ddy = C.ys[e] - yjl + (float)((long long)(uint32_t)key - cy) * cellf;
      const float d2f = ddx * ddx + ddy * ddy;
      if (d2f > hi2) continue;
      const int q = C.cidx[e];
      if (q == j) continue;
      if (d2f >= lo2) {  // near the radius: decide in double
        const double gx = __dsub_rn(C.x[q], xj), gy = __dsub_rn(C.y[q], yj);
        if (!(__dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy)) <= r2)) continue;
      }
      if (!f(q)) return;
    }
  }
}

// Cell-relative float coordinates of each sorted entry.
__global__ void k_cl_local(const tx_clusterer C, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int q = C.cidx[e];
  const unsigned long long key = C.ckey[e];
  C.xs[e] = (float)(C.x[q] - (double)(key >> 32) * C.cell);
  C.ys[e] = (float)(C.y[q] - (double)(uint32_t)key * C.cell);
}

__global__ void k_cl_core(const tx_clusterer C, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int cnt = 0;
  for_neighbours(C, n, j, [&](int) { return ++cnt <= C.k; });  // stop once core
  C.core[j] = cnt > C.k;
  C.parent[j] = j;
  C.cnt[j] = 0;
  C.rep[j] = 0ull;
  C.dlo[j] = INT32_MAX;
  C.dhi[j] = INT32_MIN;
  C.tlo[j] = INT32_MAX;
  C.thi[j] = INT32_MIN;
}

__device__ __forceinline__ int cl_find(int32_t* parent, int x) {
  volatile int32_t* p = parent;
  int px = p[x];
  while (px != x) {
    const int gp = p[px];
    if (gp != px) p[x] = gp;  // path halving: always an ancestor of x
    x = px;
    px = p[x];
  }
  return x;
}

__global__ void k_cl_union(const tx_clusterer C, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n || !C.core[j]) return;
  for_neighbours(C, n, j, [&](int q) {
    if (q >= j || !C.core[q]) return true;  // each core pair once
    int a = cl_find(C.parent, j);
    if (((volatile int32_t*)C.parent)[q] == a) return true;  // already joined
    int b = cl_find(C.parent, q);
    while (a != b) {
      if (a < b) { const int t = a; a = b; b = t; }
      // link the larger root a under the smaller root b
      const int old = atomicCAS(C.parent + a, a, b);
      if (old == a) break;
      a = cl_find(C.parent, a);
      b = cl_find(C.parent, b);
    }
    return true;
  });
}

__global__ void k_cl_label_core(const tx_clusterer C, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  C.label[j] = C.core[j] ? cl_find(C.parent, j) : -1;
}

__global__ void k_cl_label_border(const tx_clusterer C, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n || C.core[j]) return;
  int best = INT32_MAX;
  for_neighbours(C, n, j, [&](int q) {
    if (C.core[q]) best = min(best, C.label[q]);
    return true;
  });
  C.label[j] = best == INT32_MAX ? -1 : best;
}

__device__ __forceinline__ uint32_t ordered(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void k_cl_reduce(const tx_clusterer C, const tx_cand* __restrict__ c, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int l = C.label[j];
  if (l < 0) return;
  const tx_cand r = c[C.perm[j]];
  atomicAdd(C.cnt + l, 1);
  atomicMax(C.rep + l, ((unsigned long long)ordered(r.snr) << 32) | (uint32_t)(~(uint32_t)j));
  atomicMin(C.dlo + l, r.dm_index);
  atomicMax(C.dhi + l, r.dm_index);
  atomicMin(C.tlo + l, r.t);
  atomicMax(C.thi + l, r.t);
}

__global__ void k_cl_flag(const tx_clusterer C, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  C.flag[j] = C.core[j] && C.label[j] == j;
}

__global__ void k_cl_emit(const tx_clusterer C, const tx_cand* __restrict__ c, int n, tx_cluster* out,
                          int64_t* nclusters, int32_t* labels_out, int32_t* order_out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  if (labels_out) labels_out[j] = C.label[j];
  if (order_out) order_out[j] = C.perm[j];
  if (j == n - 1) *nclusters = (int64_t)C.pos[j] + C.flag[j];
  if (!C.flag[j]) return;
  const unsigned long long rk = C.rep[j];
  const int best = (int)(~(uint32_t)(rk & 0xFFFFFFFFull));
  const tx_cand r = c[C.perm[best]];
  tx_cluster o;
  o.id = j;
  o.dm_index = r.dm_index;
  o.t = r.t;
  o.w_index = r.w_index;
  o.snr = r.snr;
  o.members = C.cnt[j];
  o.dm_lo = C.dlo[j];
  o.dm_hi = C.dhi[j];
  o.t_lo = C.tlo[j];
  o.t_hi = C.thi[j];
  out[C.pos[j]] = o;
}

template <typename T>
int dalloc(T** p, int64_t n) {
  TX_CUDA(cudaMalloc((void**)p, (size_t)std::max<int64_t>(n, 1) * sizeof(T)));
  return TX_OK;
}

}  // namespace

extern "C" {

int32_t tx_clusterer_create(const tx_plan* p, double radius_ms, int32_t k, int64_t max_points, tx_clusterer** out) {
  if (!p || !out) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!(radius_ms > 0.0) || k < 0 || max_points < 1 || max_points >= INT32_MAX) {
    set_error("need radius_ms > 0, k >= 0 and 1 <= max_points < 2^31");
    return TX_ERR_INVALID_ARG;
  }
  tx_clusterer* C = new (std::nothrow) tx_clusterer();
  if (!C) { set_error("out of host memory"); return TX_ERR_OOM; }
  cudaGetDevice(&C->device);
  C->r = radius_ms;
  C->cell = radius_ms * (1.0 + 1e-9);  // a neighbour within r is never two cells away
  C->tsamp_ms = p->tsamp * 1e3;
  C->k = k;
  C->cap = max_points;
  C->ndm = p->ndm;
  const int64_t n = max_points;
  int rc = TX_OK;
  if (!rc) rc = dalloc(&C->table, p->ndm);
  if (!rc) rc = dalloc(&C->key_a, n);
  if (!rc) rc = dalloc(&C->key_b, n);
  if (!rc) rc = dalloc(&C->val_a, n);
  if (!rc) rc = dalloc(&C->val_b, n);
  if (!rc) rc = dalloc(&C->x, n);
  if (!rc) rc = dalloc(&C->y, n);
  if (!rc) rc = dalloc(&C->core, n);
  if (!rc) rc = dalloc(&C->parent, n);
  if (!rc) rc = dalloc(&C->label, n);
  if (!rc) rc = dalloc(&C->cnt, n);
  if (!rc) rc = dalloc(&C->rep, n);
  if (!rc) rc = dalloc(&C->dlo, n);
  if (!rc) rc = dalloc(&C->dhi, n);
  if (!rc) rc = dalloc(&C->tlo, n);
  if (!rc) rc = dalloc(&C->thi, n);
  if (!rc) rc = dalloc(&C->flag, n);
  if (!rc) rc = dalloc(&C->pos, n);
  if (!rc) rc = dalloc(&C->xs, n);
  if (!rc) rc = dalloc(&C->ys, n);
  if (!rc && cudaMemcpy(C->table, p->delay_ms.data(), p->delay_ms.size() * sizeof(double),
                        cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("delay table upload failed");
    rc = TX_ERR_CUDA;
  }
  if (!rc) {
    size_t a = 0, b = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, a, C->key_a, C->key_b, C->val_a, C->val_b, (int)n);
    cub::DeviceScan::ExclusiveSum(nullptr, b, C->flag, C->pos, (int)n);
    C->temp_bytes = std::max(a, b);
    if (cudaMalloc(&C->temp, std::max<size_t>(C->temp_bytes, 16)) != cudaSuccess) {
      set_error("clusterer scratch allocation failed");
      rc = TX_ERR_OOM;
    }
  }
  if (rc) { tx_clusterer_destroy(C); return rc; }
  *out = C;
  return TX_OK;
}

int32_t tx_cluster_run(tx_clusterer* C, const tx_cand* d_cands, int64_t n, tx_cluster* d_out, int64_t* d_nclusters,
                       int32_t* d_labels, int32_t* d_order, void* stream) {
  if (!C || (!d_cands && n > 0) || !d_out || !d_nclusters) { set_error("null argument"); return TX_ERR_INVALID_ARG; }
  if (n < 0 || n > C->cap) { set_error("%lld points, capacity %lld", (long long)n, (long long)C->cap); return TX_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  if (n == 0) {
    TX_CUDA(cudaMemsetAsync(d_nclusters, 0, sizeof(int64_t), st));
    return TX_OK;
  }
  const int ni = (int)n;
  const int grid = (ni + kThreads - 1) / kThreads;
  size_t tb = C->temp_bytes;
  // 1. canonical order
  k_cl_canon<<<grid, kThreads, 0, st>>>(d_cands, ni, C->key_a, C->val_a);
  TX_CUDA(cudaGetLastError());
  TX_CUDA(cub::DeviceRadixSort::SortPairs(C->temp, tb, C->key_a, C->key_b, C->val_a, C->val_b, ni, 0, 64, st));
  C->perm = C->val_b;
  // 2. coordinates and cells
  k_cl_coords<<<grid, kThreads, 0, st>>>(d_cands, C->perm, ni, C->table, C->tsamp_ms, C->cell, C->x, C->y,
                                         C->key_a, C->val_a);
  TX_CUDA(cudaGetLastError());
  unsigned long long* ck = C->key_b;       // canonical keys are no longer needed
  int32_t* ci = reinterpret_cast<int32_t*>(C->flag);
  tb = C->temp_bytes;
  TX_CUDA(cub::DeviceRadixSort::SortPairs(C->temp, tb, C->key_a, ck, C->val_a, ci, ni, 0, 64, st));
  C->ckey = ck;
  C->cidx = ci;
  k_cl_local<<<grid, kThreads, 0, st>>>(*C, ni);
  // 3-5. core flags, union-find, labels
  k_cl_core<<<grid, kThreads, 0, st>>>(*C, ni);
  k_cl_union<<<grid, kThreads, 0, st>>>(*C, ni);
  k_cl_label_core<<<grid, kThreads, 0, st>>>(*C, ni);
  k_cl_label_border<<<grid, kThreads, 0, st>>>(*C, ni);
  TX_CUDA(cudaGetLastError());
  // 6. per-cluster reductions
  k_cl_reduce<<<grid, kThreads, 0, st>>>(*C, d_cands, ni);
  // 7. clusters in id order
  int32_t* fl = C->val_a;                  // cell values are no longer needed
  tx_clusterer Cf = *C;
  Cf.flag = fl;
  k_cl_flag<<<grid, kThreads, 0, st>>>(Cf, ni);
  tb = C->temp_bytes;
  TX_CUDA(cub::DeviceScan::ExclusiveSum(C->temp, tb, fl, C->pos, ni, st));
  k_cl_emit<<<grid, kThreads, 0, st>>>(Cf, d_cands, ni, d_out, d_nclusters, d_labels, d_order);
  TX_CUDA(cudaGetLastError());
  return TX_OK;
}

void tx_clusterer_destroy(tx_clusterer* C) {
  if (!C) return;
  int prev = 0;
  cudaGetDevice(&prev);
  if (C->device >= 0) cudaSetDevice(C->device);
  for (void* q : {(void*)C->table, (void*)C->key_a, (void*)C->key_b, (void*)C->val_a, (void*)C->val_b, (void*)C->x,
                  (void*)C->y, (void*)C->core, (void*)C->parent, (void*)C->label, (void*)C->cnt, (void*)C->rep,
                  (void*)C->dlo, (void*)C->dhi, (void*)C->tlo, (void*)C->thi, (void*)C->flag, (void*)C->pos,
                  (void*)C->xs, (void*)C->ys, C->temp})
    cudaFree(q);
  cudaSetDevice(prev);
  delete C;
}

}  // extern "C"
