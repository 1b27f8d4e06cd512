// Sparse front end (Sec. 2.2; Sec. 3.2 and 3.3): diagonal boosting by a
// maximum-product matching, Cuthill-McKee bandwidth reduction, assembly of
// the reordered matrix into the dense band storage, and the permutations of
// right-hand sides and solutions.  See include/sap_sparse.h.
//
// GPU: the matching weights (S1), the scale factors (S4), the bandwidth, the
// band assembly and the permutations.  Host (as in the paper, whose graph
// searches run on the CPU): the initial match (S2), the shortest augmenting
// paths (S3), the level structure and the Cuthill-McKee order.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <limits>
#include <queue>
#include <vector>
#include <atomic>
#include <thread>
#include "sap_sparse.h"
#include "sap_blocks.h"
#include "sap_internal.cuh"

namespace {

constexpr double kInf = std::numeric_limits<double>::infinity();

#define CKS(x)                                              \
  do {                                                      \
    if ((x) != cudaSuccess) { cudaGetLastError(); return SAP_ERR_CUDA; } \
  } while (0)

// ---- kernels ----

// S1: a_i = max_j |a_ij| (one warp per row) and c_ij = log a_i - log |a_ij|,
// infinite for a stored zero.
__global__ void k_db_weights(int64_t n, const int64_t* __restrict__ rowptr, const double* __restrict__ val,
                             double* __restrict__ a, double* __restrict__ c) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const int64_t lo = rowptr[i], hi = rowptr[i + 1];
  double m = 0.0;
  for (int64_t p = lo + lane; p < hi; p += 32) m = fmax(m, fabs(val[p]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) a[i] = m;
  const double lm = log(m);
  for (int64_t p = lo + lane; p < hi; p += 32) c[p] = val[p] != 0.0 ? lm - log(fabs(val[p])) : kInf;
}

// S4: r_i = exp(u_i) / a_i, s_j = exp(v_j).
__global__ void k_db_scale(int64_t n, const double* __restrict__ a, const double* __restrict__ u,
                           const double* __restrict__ v, double* __restrict__ r, double* __restrict__ s) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  r[i] = exp(u[i]) / a[i];
  s[i] = exp(v[i]);
}

__global__ void k_perm_compose(int64_t n, const int32_t* __restrict__ outer, const int32_t* __restrict__ inner,
                               int32_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = outer[inner[i]];
}

// max |rownew[i] - colnew[j]| over the stored entries (one warp per row).
__global__ void k_bandwidth(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const int32_t* __restrict__ rownew, const int32_t* __restrict__ colnew,
                            int* __restrict__ K) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const int64_t I = rownew ? rownew[i] : i;
  int64_t m = 0;
  for (int64_t p = rowptr[i] + lane; p < rowptr[i + 1]; p += 32) {
    const int64_t J = colnew ? colnew[col[p]] : col[p];
    m = max(m, I > J ? I - J : J - I);
  }
  int mi = (int)m;
  for (int o = 16; o > 0; o >>= 1) mi = max(mi, __shfl_xor_sync(0xffffffffu, mi, o));
  if (lane == 0 && mi > 0) atomicMax(K, mi);
}

// band[(K + I - J) * n + J] = (r_i a_ij) s_j; an entry outside the band is
// dropped (drop) or sets *bad.
__global__ void k_to_band(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                          const double* __restrict__ val, const int32_t* __restrict__ rownew,
                          const int32_t* __restrict__ colnew, const double* __restrict__ r,
                          const double* __restrict__ s, int K, bool drop, double* __restrict__ band,
                          int* __restrict__ bad) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const int64_t I = rownew ? rownew[i] : i;
  for (int64_t p = rowptr[i] + lane; p < rowptr[i + 1]; p += 32) {
    const int64_t j = col[p];
    const int64_t J = colnew ? colnew[j] : j;
    const int64_t dd = K + I - J;
    if (dd < 0 || dd > 2 * K) {
      if (!drop) atomicExch(bad, 1);
      continue;
    }
    double x = val[p];
    if (r) x = (r[i] * x) * s[j];
    band[dd * n + J] = x;
  }
}

// y[rownew[i]] = sum_p ((r_i a_ip) s_j) x[colnew[j]], j = col[p]: the
// reordered operator's row; one warp per stored row, partial sums combined
// by shuffles.
__global__ void k_spmv_pcsr(sap::CsrOp A, const double* __restrict__ x, double* __restrict__ y, sap::Gate gt) {
  if (sap::gate_skip(gt)) return;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= A.n) return;
  const double ri = A.r ? A.r[i] : 1.0;
  double acc = 0.0;
  for (int64_t p = A.rowptr[i] + lane; p < A.rowptr[i + 1]; p += 32) {
    const int32_t j = A.col[p];
    const double e = A.r ? (ri * A.val[p]) * A.s[j] : A.val[p];
    acc += e * x[A.colnew ? A.colnew[j] : j];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) y[A.rownew ? A.rownew[i] : i] = acc;
}

// w[dist] += |(r_i a_ij) s_j| over the stored entries, dist = |I - J| <= K
// (a per-CTA histogram in shared memory, then one atomic per bin).
__global__ void k_dist_weights(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const double* __restrict__ val, const int32_t* __restrict__ rownew,
                               const int32_t* __restrict__ colnew, const double* __restrict__ r,
                               const double* __restrict__ s, int K, double* __restrict__ w) {
  extern __shared__ double hist[];
  for (int t = threadIdx.x; t <= K; t += blockDim.x) hist[t] = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const int64_t I = rownew ? rownew[i] : i;
    for (int64_t p = rowptr[i] + lane; p < rowptr[i + 1]; p += 32) {
      const int64_t j = col[p];
      const int64_t J = colnew ? colnew[j] : j;
      const int64_t dd = I > J ? I - J : J - I;
      const double e = r ? fabs((r[i] * val[p]) * s[j]) : fabs(val[p]);
      if (dd <= K) atomicAdd(&hist[dd], e);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t <= K; t += blockDim.x)
    if (hist[t] != 0.0) atomicAdd(&w[t], hist[t]);
}

__global__ void k_permute_rhs(int64_t n, const double* __restrict__ b, const int32_t* __restrict__ rownew,
                              const double* __restrict__ r, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[rownew[i]] = r ? r[i] * b[i] : b[i];
}

__global__ void k_unpermute(int64_t n, const double* __restrict__ y, const int32_t* __restrict__ colnew,
                            const double* __restrict__ s, double* __restrict__ x) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) x[j] = s ? s[j] * y[colnew[j]] : y[colnew[j]];
}

unsigned blocks_for(int64_t threads, int per) { return (unsigned)((threads + per - 1) / per); }

// Device buffer released on scope exit.
template <typename T>
struct DevBuf {
  T* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
  bool alloc(size_t n) { return cudaMalloc(&p, (n ? n : 1) * sizeof(T)) == cudaSuccess; }
};

// ---- host: matching (S2, S3) ----

// Minimum perfect matching on the CSR graph with weights c: returns false
// when none exists.  Potentials u (rows), v (columns) with
// c_ij - u_i - v_j >= 0 on every edge and = 0 on the matching.
bool min_matching(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                  const std::vector<double>& c, std::vector<int32_t>& col_of_row, std::vector<double>& u,
                  std::vector<double>& v) {
  u.assign(n, kInf);
  v.assign(n, kInf);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) u[i] = std::min(u[i], c[p]);
  for (int64_t i = 0; i < n; ++i) {
    if (u[i] == kInf) return false;                    // a row without a usable entry
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
      if (c[p] != kInf) v[ci[p]] = std::min(v[ci[p]], c[p] - u[i]);
  }
  for (int64_t j = 0; j < n; ++j)
    if (v[j] == kInf) return false;                    // a column without a usable entry
  // S2: match along zero reduced cost, rows in order, first free column
  col_of_row.assign(n, -1);
  std::vector<int32_t> row_of_col(n, -1);
  std::vector<double> mcost(n, 0.0);                  // c of each row's matched edge
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int32_t j = ci[p];
      if (c[p] != kInf && row_of_col[j] < 0 && c[p] - u[i] - v[j] == 0.0) {
        row_of_col[j] = (int32_t)i;
        col_of_row[i] = j;
        mcost[i] = c[p];
        break;
      }
    }
  // S3: a Dijkstra search on the reduced costs from every unmatched row
  std::vector<double> dist(n, kInf), pcost(n, 0.0);
  std::vector<int32_t> pred(n, -1);
  std::vector<char> done(n, 0);
  std::vector<int32_t> touched, scanned;
  using Item = std::pair<double, int32_t>;
  for (int64_t i0 = 0; i0 < n; ++i0) {
    if (col_of_row[i0] >= 0) continue;
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
    touched.clear();
    scanned.clear();
    auto relax = [&](int64_t i, double base) {
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        const int32_t j = ci[p];
        if (c[p] == kInf || done[j]) continue;
        const double d = base + (c[p] - u[i] - v[j]);
        if (d < dist[j]) {
          if (dist[j] == kInf) touched.push_back(j);
          dist[j] = d;
          pred[j] = (int32_t)i;
          pcost[j] = c[p];
          heap.push({d, j});
        }
      }
    };
    relax(i0, 0.0);
    int32_t jfree = -1;
    double D = kInf;
    while (!heap.empty()) {
      const Item t = heap.top();
      heap.pop();
      const int32_t j = t.second;
      if (done[j] || t.first > dist[j]) continue;
      done[j] = 1;
      scanned.push_back(j);
      if (row_of_col[j] < 0) {
        jfree = j;
        D = t.first;
        break;
      }
      relax(row_of_col[j], t.first);
    }
    if (jfree < 0) return false;
    // potentials: v_j += dist_j - D on the scanned columns, then each row on
    // them (and i0) takes u_i = c(i, its column) - v(its column)
    for (int32_t j : scanned) v[j] += dist[j] - D;
    for (int32_t j = jfree;;) {                        // flip the augmenting path
      const int32_t i = pred[j];
      const int32_t jprev = col_of_row[i];
      col_of_row[i] = j;
      row_of_col[j] = i;
      mcost[i] = pcost[j];
      if (i == i0) break;
      j = jprev;
    }
    for (int32_t j : scanned) {
      const int32_t i = row_of_col[j];
      u[i] = mcost[i] - v[j];
    }
    for (int32_t j : touched) {
      dist[j] = kInf;
      done[j] = 0;
    }
  }
  return true;
}

// ---- host: Cuthill-McKee ----

constexpr int kCmMaxStarts = 5;

// perm[old] = new for the neighbour lists (CSR: nb_ptr, nb).
void cm_order(int64_t n, const std::vector<int64_t>& nb_ptr, const std::vector<int32_t>& nb,
              std::vector<int32_t>& perm) {
  std::vector<int64_t> deg(n);
  for (int64_t x = 0; x < n; ++x) deg[x] = nb_ptr[x + 1] - nb_ptr[x];
  auto less = [&](int32_t a, int32_t b) { return deg[a] < deg[b] || (deg[a] == deg[b] && a < b); };
  std::vector<char> placed(n, 0);       // in an ordered component
  std::vector<int32_t> mark(n, -1);     // BFS trial stamp
  std::vector<char> tried(n, 0);
  std::vector<int32_t> order;
  order.reserve(n);
  std::vector<int32_t> by_key(n);       // nodes by (degree, index): the next component's start
  for (int64_t x = 0; x < n; ++x) by_key[x] = (int32_t)x;
  std::sort(by_key.begin(), by_key.end(), less);
  size_t next_start = 0;
  int32_t stamp = 0;
  std::vector<int32_t> cur, nxt, last;
  // BFS levels from s over unplaced nodes: height, widest level, last level
  auto levels = [&](int32_t s, int64_t& height, int64_t& width) {
    ++stamp;
    cur.assign(1, s);
    mark[s] = stamp;
    height = 0;
    width = 0;
    while (!cur.empty()) {
      ++height;
      width = std::max<int64_t>(width, (int64_t)cur.size());
      last = cur;
      nxt.clear();
      for (int32_t x : cur)
        for (int64_t p = nb_ptr[x]; p < nb_ptr[x + 1]; ++p) {
          const int32_t y = nb[p];
          if (!placed[y] && mark[y] != stamp) {
            mark[y] = stamp;
            nxt.push_back(y);
          }
        }
      cur.swap(nxt);
    }
  };
  std::vector<int32_t> tried_list;
  while (order.size() < (size_t)n) {
    while (placed[by_key[next_start]]) ++next_start;
    int32_t s = by_key[next_start];
    int32_t best = -1;
    int64_t bh = 0, bw = 0;
    tried_list.clear();
    for (int t = 0; t < kCmMaxStarts; ++t) {
      int64_t h, w;
      levels(s, h, w);
      if (best < 0 || (h > bh && w < bw)) {
        best = s;
        bh = h;
        bw = w;
      } else {
        break;
      }
      tried[s] = 1;
      tried_list.push_back(s);
      int32_t cand = -1;
      for (int32_t y : last)
        if (!tried[y] && (cand < 0 || less(y, cand))) cand = y;
      if (cand < 0) break;
      s = cand;
    }
    for (int32_t x : tried_list) tried[x] = 0;
    // the ordering: BFS from the best start, neighbours by (degree, index)
    const size_t base = order.size();
    order.push_back(best);
    placed[best] = 1;
    std::vector<int32_t> add;
    for (size_t k = base; k < order.size(); ++k) {
      const int32_t x = order[k];
      add.clear();
      for (int64_t p = nb_ptr[x]; p < nb_ptr[x + 1]; ++p)
        if (!placed[nb[p]]) add.push_back(nb[p]);
      std::sort(add.begin(), add.end(), less);
      for (int32_t y : add) {
        placed[y] = 1;
        order.push_back(y);
      }
    }
  }
  perm.resize(n);
  for (int64_t k = 0; k < n; ++k) perm[order[k]] = (int32_t)k;
}

bool valid_csr_args(int64_t n, int64_t nnz, const void* rowptr, const void* col) {
  return n >= 1 && n < (int64_t(1) << 31) && nnz >= 0 && rowptr && col;
}

}  // namespace

extern "C" sap_status_t sap_db_reorder(int64_t n, int64_t nnz, const int64_t* rowptr_dev, const int32_t* col_dev,
                                       const double* val_dev, int32_t* rownew_dev, double* rscale_dev,
                                       double* cscale_dev, double* logprod, cudaStream_t stream) {
  if (!valid_csr_args(n, nnz, rowptr_dev, col_dev) || !val_dev || !rownew_dev) return SAP_ERR_INVALID_ARG;
  if ((rscale_dev == nullptr) != (cscale_dev == nullptr)) return SAP_ERR_INVALID_ARG;
  DevBuf<double> a, c;
  if (!a.alloc(n) || !c.alloc(nnz)) return SAP_ERR_OOM;
  sap::count_launches(1);
  k_db_weights<<<blocks_for(n * 32, 256), 256, 0, stream>>>(n, rowptr_dev, val_dev, a.p, c.p);
  CKS(cudaGetLastError());
  std::vector<int64_t> rp(n + 1);
  std::vector<int32_t> ci(nnz);
  std::vector<double> ch(nnz), vh;
  CKS(cudaMemcpyAsync(rp.data(), rowptr_dev, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
  CKS(cudaMemcpyAsync(ci.data(), col_dev, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
  CKS(cudaMemcpyAsync(ch.data(), c.p, nnz * sizeof(double), cudaMemcpyDeviceToHost, stream));
  if (logprod) {
    vh.resize(nnz);
    CKS(cudaMemcpyAsync(vh.data(), val_dev, nnz * sizeof(double), cudaMemcpyDeviceToHost, stream));
  }
  CKS(cudaStreamSynchronize(stream));
  if (rp[0] != 0 || rp[n] != nnz) return SAP_ERR_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i)
    if (rp[i + 1] <= rp[i]) return SAP_ERR_INVALID_ARG;
  for (int64_t p = 0; p < nnz; ++p)
    if (ci[p] < 0 || ci[p] >= n) return SAP_ERR_INVALID_ARG;
  std::vector<int32_t> col_of_row;
  std::vector<double> u, v;
  if (!min_matching(n, rp, ci, ch, col_of_row, u, v)) return SAP_ERR_SINGULAR;
  CKS(cudaMemcpyAsync(rownew_dev, col_of_row.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
  if (rscale_dev) {
    DevBuf<double> ud, vd;
    if (!ud.alloc(n) || !vd.alloc(n)) return SAP_ERR_OOM;
    CKS(cudaMemcpyAsync(ud.p, u.data(), n * sizeof(double), cudaMemcpyHostToDevice, stream));
    CKS(cudaMemcpyAsync(vd.p, v.data(), n * sizeof(double), cudaMemcpyHostToDevice, stream));
    sap::count_launches(1);
    k_db_scale<<<blocks_for(n, 256), 256, 0, stream>>>(n, a.p, ud.p, vd.p, rscale_dev, cscale_dev);
    CKS(cudaGetLastError());
    CKS(cudaStreamSynchronize(stream));           // before ud, vd are freed
  }
  if (logprod) {
    double lp = 0.0;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
        if (ci[p] == col_of_row[i]) lp += std::log(std::fabs(vh[p]));
    *logprod = lp;
  }
  CKS(cudaStreamSynchronize(stream));
  return SAP_OK;
}

extern "C" sap_status_t sap_cm_reorder(int64_t n, int64_t nnz, const int64_t* rowptr_dev, const int32_t* col_dev,
                                       const int32_t* rownew_dev, int32_t* perm_dev, int32_t* K_out,
                                       cudaStream_t stream) {
  if (!valid_csr_args(n, nnz, rowptr_dev, col_dev) || !perm_dev) return SAP_ERR_INVALID_ARG;
  std::vector<int64_t> rp(n + 1);
  std::vector<int32_t> ci(nnz), rn;
  CKS(cudaMemcpyAsync(rp.data(), rowptr_dev, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
  CKS(cudaMemcpyAsync(ci.data(), col_dev, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
  if (rownew_dev) {
    rn.resize(n);
    CKS(cudaMemcpyAsync(rn.data(), rownew_dev, n * sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
  }
  CKS(cudaStreamSynchronize(stream));
  if (rp[0] != 0 || rp[n] != nnz) return SAP_ERR_INVALID_ARG;
  for (int64_t p = 0; p < nnz; ++p)
    if (ci[p] < 0 || ci[p] >= n) return SAP_ERR_INVALID_ARG;
  // pattern of B + B^T without self loops: both directions of every entry,
  // sorted and made unique per node
  std::vector<int64_t> cnt(n + 1, 0);
  for (int64_t i = 0; i < n; ++i) {
    const int32_t r = rownew_dev ? rn[i] : (int32_t)i;
    if (r < 0 || r >= n) return SAP_ERR_INVALID_ARG;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] != r) {
        ++cnt[r + 1];
        ++cnt[ci[p] + 1];
      }
  }
  for (int64_t x = 0; x < n; ++x) cnt[x + 1] += cnt[x];
  std::vector<int32_t> adj(cnt[n]);
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  for (int64_t i = 0; i < n; ++i) {
    const int32_t r = rownew_dev ? rn[i] : (int32_t)i;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] != r) {
        adj[fill[r]++] = ci[p];
        adj[fill[ci[p]]++] = r;
      }
  }
  std::vector<int64_t> nb_ptr(n + 1, 0);
  std::vector<int32_t> nb;
  nb.reserve(adj.size());
  for (int64_t x = 0; x < n; ++x) {
    auto b = adj.begin() + cnt[x], e = adj.begin() + cnt[x + 1];
    std::sort(b, e);
    e = std::unique(b, e);
    nb.insert(nb.end(), b, e);
    nb_ptr[x + 1] = (int64_t)nb.size();
  }
  std::vector<int32_t> perm;
  cm_order(n, nb_ptr, nb, perm);
  CKS(cudaMemcpyAsync(perm_dev, perm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
  if (K_out) {
    int64_t K = 0;
    for (int64_t i = 0; i < n; ++i) {
      const int64_t I = perm[rownew_dev ? rn[i] : (int32_t)i];
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) K = std::max<int64_t>(K, std::llabs(I - (int64_t)perm[ci[p]]));
    }
    *K_out = (int32_t)K;
  }
  CKS(cudaStreamSynchronize(stream));
  return SAP_OK;
}

// The third-stage reordering (include/sap_blocks.h): CM of every block's
// A_i + A_i^T on its own, from a host copy of the band.
extern "C" sap_status_t sap_block_cm_reorder(const double* band_dev, int64_t N, int32_t K, int32_t P,
                                             int32_t* perm_dev, int32_t* Ki_host, cudaStream_t stream) {
  if (!band_dev || !perm_dev || N < 1 || K < 1 || P < 1 || N < P || N >= (int64_t(1) << 31)) return SAP_ERR_INVALID_ARG;
  const int64_t W = 2 * (int64_t)K + 1;
  std::vector<double> band;
  std::vector<int32_t> perm_all;
  try {
    band.resize((size_t)(W * N));
    perm_all.resize((size_t)N);
  } catch (...) {
    return SAP_ERR_OOM;
  }
  CKS(cudaMemcpyAsync(band.data(), band_dev, (size_t)(W * N) * sizeof(double), cudaMemcpyDeviceToHost, stream));
  CKS(cudaStreamSynchronize(stream));
  // the partition of sap_factor: the first N mod P blocks have one row more
  const int64_t q = N / P, pr = N - (int64_t)P * q;
  std::vector<int64_t> off((size_t)P + 1, 0);
  for (int b = 0; b < P; ++b) off[(size_t)b + 1] = off[(size_t)b] + q + (b < pr ? 1 : 0);
  std::vector<int32_t> Kb((size_t)P, 0);
  // one block's pattern of A_b + A_b^T and its CM order; blocks are independent
  // (the paper runs this stage in parallel for every A_i), each worker writes
  // only its own blocks' slices
  auto one_block = [&](int b) {
    const int64_t s = off[(size_t)b], n = off[(size_t)b + 1] - s;
    std::vector<int64_t> nb_ptr((size_t)(n + 1), 0);
    std::vector<int32_t> nb, p;
    for (int64_t a = 0; a < n; ++a) {
      const int64_t g = s + a;
      for (int64_t dq = -K; dq <= K; ++dq) {     // neighbours in ascending order
        const int64_t c = a + dq;
        if (dq == 0 || c < 0 || c >= n) continue;
        // entry (g, s+c) at band[(K - dq) N + s + c], entry (s+c, g) at band[(K + dq) N + g]
        if (band[(size_t)((K - dq) * N + s + c)] != 0.0 || band[(size_t)((K + dq) * N + g)] != 0.0)
          nb.push_back((int32_t)c);
      }
      nb_ptr[(size_t)(a + 1)] = (int64_t)nb.size();
    }
    cm_order(n, nb_ptr, nb, p);
    int64_t kb = 0;
    for (int64_t a = 0; a < n; ++a)
      for (int64_t e = nb_ptr[(size_t)a]; e < nb_ptr[(size_t)(a + 1)]; ++e)
        kb = std::max<int64_t>(kb, std::llabs((int64_t)p[(size_t)a] - p[(size_t)nb[(size_t)e]]));
    Kb[(size_t)b] = (int32_t)kb;
    std::copy(p.begin(), p.end(), perm_all.begin() + s);
  };
  const int nthreads = (int)std::max(1u, std::min<unsigned>((unsigned)P, std::min(16u, std::thread::hardware_concurrency())));
  std::atomic<int> next{0}, failed{0};
  auto worker = [&]() {
    for (int b = next++; b < P; b = next++) {
      try {
        one_block(b);
      } catch (...) {          // an allocation failed: no exception may leave a thread
        failed = 1;
      }
    }
  };
  std::vector<std::thread> pool;
  try {
    for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker);
  } catch (...) {
    // no more threads: the calling thread does the rest
  }
  worker();
  for (auto& t : pool) t.join();
  if (failed) return SAP_ERR_OOM;
  if (Ki_host)
    for (int b = 0; b < P; ++b) Ki_host[b] = Kb[(size_t)b];
  CKS(cudaMemcpyAsync(perm_dev, perm_all.data(), (size_t)N * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
  CKS(cudaStreamSynchronize(stream));
  return SAP_OK;
}

extern "C" sap_status_t sap_perm_compose(int64_t n, const int32_t* outer_dev, const int32_t* inner_dev,
                                         int32_t* out_dev, cudaStream_t stream) {
  if (n < 1 || !outer_dev || !inner_dev || !out_dev) return SAP_ERR_INVALID_ARG;
  sap::count_launches(1);
  k_perm_compose<<<blocks_for(n, 256), 256, 0, stream>>>(n, outer_dev, inner_dev, out_dev);
  CKS(cudaGetLastError());
  return SAP_OK;
}

extern "C" sap_status_t sap_sparse_bandwidth(int64_t n, int64_t nnz, const int64_t* rowptr_dev,
                                             const int32_t* col_dev, const int32_t* rownew_dev,
                                             const int32_t* colnew_dev, int32_t* K_out, cudaStream_t stream) {
  if (!valid_csr_args(n, nnz, rowptr_dev, col_dev) || !K_out) return SAP_ERR_INVALID_ARG;
  DevBuf<int> Kd;
  if (!Kd.alloc(1)) return SAP_ERR_OOM;
  CKS(cudaMemsetAsync(Kd.p, 0, sizeof(int), stream));
  sap::count_launches(1);
  k_bandwidth<<<blocks_for(n * 32, 256), 256, 0, stream>>>(n, rowptr_dev, col_dev, rownew_dev, colnew_dev, Kd.p);
  CKS(cudaGetLastError());
  int K = 0;
  CKS(cudaMemcpyAsync(&K, Kd.p, sizeof(int), cudaMemcpyDeviceToHost, stream));
  CKS(cudaStreamSynchronize(stream));
  *K_out = K;
  return SAP_OK;
}

extern "C" sap_status_t sap_sparse_to_band(int64_t n, int64_t nnz, const int64_t* rowptr_dev,
                                           const int32_t* col_dev, const double* val_dev, const int32_t* rownew_dev,
                                           const int32_t* colnew_dev, const double* rscale_dev,
                                           const double* cscale_dev, int32_t K, int32_t drop, double* band_dev,
                                           cudaStream_t stream) {
  if (!valid_csr_args(n, nnz, rowptr_dev, col_dev) || !val_dev || !band_dev || K < 0 || K >= n)
    return SAP_ERR_INVALID_ARG;
  if ((rscale_dev == nullptr) != (cscale_dev == nullptr)) return SAP_ERR_INVALID_ARG;
  DevBuf<int> bad;
  if (!bad.alloc(1)) return SAP_ERR_OOM;
  CKS(cudaMemsetAsync(bad.p, 0, sizeof(int), stream));
  CKS(cudaMemsetAsync(band_dev, 0, (size_t)(2 * K + 1) * n * sizeof(double), stream));
  sap::count_launches(1);
  k_to_band<<<blocks_for(n * 32, 256), 256, 0, stream>>>(n, rowptr_dev, col_dev, val_dev, rownew_dev, colnew_dev,
                                                          rscale_dev, cscale_dev, K, drop != 0, band_dev,
                                                          bad.p);
  CKS(cudaGetLastError());
  int b = 0;
  CKS(cudaMemcpyAsync(&b, bad.p, sizeof(int), cudaMemcpyDeviceToHost, stream));
  CKS(cudaStreamSynchronize(stream));
  return b ? SAP_ERR_INVALID_ARG : SAP_OK;
}

extern "C" sap_status_t sap_sparse_permute_rhs(int64_t n, const double* b_dev, const int32_t* rownew_dev,
                                               const double* rscale_dev, double* out_dev, cudaStream_t stream) {
  if (n < 1 || !b_dev || !rownew_dev || !out_dev || b_dev == out_dev) return SAP_ERR_INVALID_ARG;
  sap::count_launches(1);
  k_permute_rhs<<<blocks_for(n, 256), 256, 0, stream>>>(n, b_dev, rownew_dev, rscale_dev, out_dev);
  CKS(cudaGetLastError());
  return SAP_OK;
}

extern "C" sap_status_t sap_sparse_unpermute_solution(int64_t n, const double* y_dev, const int32_t* colnew_dev,
                                                      const double* cscale_dev, double* x_dev,
                                                      cudaStream_t stream) {
  if (n < 1 || !y_dev || !colnew_dev || !x_dev || y_dev == x_dev) return SAP_ERR_INVALID_ARG;
  sap::count_launches(1);
  k_unpermute<<<blocks_for(n, 256), 256, 0, stream>>>(n, y_dev, colnew_dev, cscale_dev, x_dev);
  CKS(cudaGetLastError());
  return SAP_OK;
}

extern "C" sap_status_t sap_sparse_drop_bandwidth(int64_t n, int64_t nnz, const int64_t* rowptr_dev,
                                                  const int32_t* col_dev, const double* val_dev,
                                                  const int32_t* rownew_dev, const int32_t* colnew_dev,
                                                  const double* rscale_dev, const double* cscale_dev, int32_t K,
                                                  double frac, int32_t* Kdrop_out, cudaStream_t stream) {
  if (!valid_csr_args(n, nnz, rowptr_dev, col_dev) || !val_dev || !Kdrop_out || K < 0 || K >= n || !(frac >= 0.0))
    return SAP_ERR_INVALID_ARG;
  if ((rscale_dev == nullptr) != (cscale_dev == nullptr)) return SAP_ERR_INVALID_ARG;
  DevBuf<double> w;
  if (!w.alloc((size_t)K + 1)) return SAP_ERR_OOM;
  CKS(cudaMemsetAsync(w.p, 0, ((size_t)K + 1) * sizeof(double), stream));
  const size_t sm = ((size_t)K + 1) * sizeof(double);
  if (sm > 48 * 1024) CKS(cudaFuncSetAttribute(k_dist_weights, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int dev = 0, sms = 1;
  CKS(cudaGetDevice(&dev));
  CKS(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  sap::count_launches(1);
  k_dist_weights<<<4 * sms, 256, sm, stream>>>(n, rowptr_dev, col_dev, val_dev, rownew_dev, colnew_dev, rscale_dev,
                                                cscale_dev, K, w.p);
  CKS(cudaGetLastError());
  std::vector<double> wh((size_t)K + 1);
  CKS(cudaMemcpyAsync(wh.data(), w.p, ((size_t)K + 1) * sizeof(double), cudaMemcpyDeviceToHost, stream));
  CKS(cudaStreamSynchronize(stream));
  double total = 0.0;
  for (int d = 0; d <= K; ++d) total += wh[d];
  // the smallest K' whose dropped tail sum_{d > K'} w[d] is at most frac * total
  int Kd = K;
  double tail = 0.0;
  while (Kd > 0 && tail + wh[Kd] <= frac * total) tail += wh[Kd--];
  *Kdrop_out = Kd;
  return SAP_OK;
}

namespace sap {
cudaError_t launch_spmv_pcsr(const CsrOp& A, const double* x, double* y, cudaStream_t s, Gate gt) {
  count_launches(1);
  k_spmv_pcsr<<<blocks_for(A.n * 32, 256), 256, 0, s>>>(A, x, y, gt);
  return cudaGetLastError();
}
}  // namespace sap

