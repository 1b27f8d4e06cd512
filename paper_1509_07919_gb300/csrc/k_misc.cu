// FP64 banded SpMV (y = A x, y = A^T x) over the band storage of Sec. 3.1,
// the band gradient -lambda x^T, and the fused FP64 vector kernels of the
// BiCGStab(2) iteration (Sleijpen & Fokkema 1993, l = 2; Sec. 2.1.1).
//
// Reductions are deterministic: a fixed grid writes one partial per block,
// and the last block to finish (atomic ticket) sums the partials in a fixed
// order and evaluates the iteration's scalar recurrences on the device, so
// the host never round-trips for alpha, beta, omega, gamma.
#include <cuda_runtime.h>
#include <cstdint>
#include "sap_internal.cuh"
#include "krylov.cuh"
#include "tc_sm103.cuh"

namespace sap {

// ------------------------------------------------------------------ SpMV --
namespace {
constexpr int SPMV_T = 128;

// y_i = sum_c band[c N + j] x_j, j = i + K - c  (A x)
// y_j = sum_c band[c N + j] x_i, i = j + c - K  (A^T x)
// x is staged in shared memory for the CTA's rows plus a K-halo each side.
// Each thread keeps 16 band loads in flight; the band is read once per
// product with evict-first loads (__ldcs), so that the Krylov vectors stay
// resident in L2 across the iteration.
template <bool TRANS>
__global__ void __launch_bounds__(SPMV_T)
k_spmv(const double* __restrict__ band, int64_t N, int K, const double* __restrict__ x,
       double* __restrict__ y, Gate gt) {
  extern __shared__ double xs[];
  if (gate_skip(gt)) return;
  const int64_t i0 = (int64_t)blockIdx.x * SPMV_T;
  const int span = SPMV_T + 2 * K;
  for (int t = threadIdx.x; t < span; t += SPMV_T) {
    int64_t j = i0 - K + t;
    xs[t] = (j >= 0 && j < N) ? x[j] : 0.0;
  }
  __syncthreads();
  const int64_t i = i0 + threadIdx.x;
  if (i >= N) return;
  const int W = 2 * K + 1;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  // local index of x_j in xs: j - (i0 - K)
  if (!TRANS) {
    // j = i + K - c; in-range j <=> c in [max(0, i+K-(N-1)), min(2K, i+K)]
    int clo = (int)max((int64_t)0, i + K - (N - 1));
    int chi = (int)min((int64_t)(W - 1), i + K);
    const double* bp = band + i + K;            // band[c N + i + K - c] = bp[c (N - 1)]
    const int64_t stride = N - 1;
    const int xl = threadIdx.x + 2 * K;         // xs index of j = i + K - c is xl - c
    int c = clo;
    for (; c + 15 <= chi; c += 16) {
      double v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) v[u] = __ldcs(bp + (int64_t)(c + u) * stride);
#pragma unroll
      for (int u = 0; u < 16; u += 4) {
        a0 += v[u] * xs[xl - c - u];
        a1 += v[u + 1] * xs[xl - c - u - 1];
        a2 += v[u + 2] * xs[xl - c - u - 2];
        a3 += v[u + 3] * xs[xl - c - u - 3];
      }
    }
    for (; c + 3 <= chi; c += 4) {
      a0 += __ldcs(bp + (int64_t)c * stride) * xs[xl - c];
      a1 += __ldcs(bp + (int64_t)(c + 1) * stride) * xs[xl - c - 1];
      a2 += __ldcs(bp + (int64_t)(c + 2) * stride) * xs[xl - c - 2];
      a3 += __ldcs(bp + (int64_t)(c + 3) * stride) * xs[xl - c - 3];
    }
    for (; c <= chi; ++c) a0 += __ldcs(bp + (int64_t)c * stride) * xs[xl - c];
  } else {
    // i' = i + c - K in range <=> c in [max(0, K-i), min(2K, N-1-i+K)]
    int clo = (int)max((int64_t)0, (int64_t)K - i);
    int chi = (int)min((int64_t)(W - 1), N - 1 - i + K);
    const double* bp = band + i;
    const int xl = threadIdx.x;                 // xs index of i + c - K is xl + c
    int c = clo;
    for (; c + 15 <= chi; c += 16) {
      double v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) v[u] = __ldcs(bp + (int64_t)(c + u) * N);
#pragma unroll
      for (int u = 0; u < 16; u += 4) {
        a0 += v[u] * xs[xl + c + u];
        a1 += v[u + 1] * xs[xl + c + u + 1];
        a2 += v[u + 2] * xs[xl + c + u + 2];
        a3 += v[u + 3] * xs[xl + c + u + 3];
      }
    }
    for (; c + 3 <= chi; c += 4) {
      a0 += __ldcs(bp + (int64_t)c * N) * xs[xl + c];
      a1 += __ldcs(bp + (int64_t)(c + 1) * N) * xs[xl + c + 1];
      a2 += __ldcs(bp + (int64_t)(c + 2) * N) * xs[xl + c + 2];
      a3 += __ldcs(bp + (int64_t)(c + 3) * N) * xs[xl + c + 3];
    }
    for (; c <= chi; ++c) a0 += __ldcs(bp + (int64_t)c * N) * xs[xl + c];
  }
  y[i] = (a0 + a1) + (a2 + a3);
}

__global__ void k_grad_band(const double* __restrict__ lam, const double* __restrict__ x, int64_t N, int K,
                            double* __restrict__ g) {
  const int64_t total = (int64_t)(2 * K + 1) * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = e / N, j = e - c * N;
    int64_t i = j + c - K;
    g[e] = (i >= 0 && i < N) ? -lam[i] * x[j] : 0.0;
  }
}
}  // namespace

cudaError_t launch_spmv(const double* band, int64_t N, int K, const double* x, double* y, bool transpose,
                        cudaStream_t s, Gate gt) {
  int64_t nb = (N + SPMV_T - 1) / SPMV_T;
  size_t smem = (SPMV_T + 2 * (size_t)K) * sizeof(double);
  cudaError_t e;
  if (transpose) {
    e = cudaFuncSetAttribute(k_spmv<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_spmv<true><<<(unsigned)nb, SPMV_T, smem, s>>>(band, N, K, x, y, gt);
  } else {
    e = cudaFuncSetAttribute(k_spmv<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_spmv<false><<<(unsigned)nb, SPMV_T, smem, s>>>(band, N, K, x, y, gt);
  }
  return cudaGetLastError();
}

cudaError_t launch_grad_band(const double* lam, const double* x, int64_t N, int K, double* g, cudaStream_t s) {
  count_launches(1);
  k_grad_band<<<152 * 8, 256, 0, s>>>(lam, x, N, K, g);
  return cudaGetLastError();
}

// --------------------------------------------------------------- Krylov --
namespace {
constexpr int RT = 256;

__device__ __forceinline__ bool kr_skip(const KrylovDev& kd) {
  Gate g;
  g.flags = kd.flags;
  g.mode = kd.gmode;
  return gate_skip(g);
}

// Block-reduce ND values; the last block to finish sums all partials and
// returns true (its thread 0 then holds the sums in red[0..ND) and runs the
// epilogue).  Every sum is taken in one fixed order (partials strided over
// the threads, a shuffle butterfly, warp sums in warp order), so results do
// not depend on block scheduling; the loads of the final sum are spread over
// the whole block rather than chained through one thread.
template <int ND>
__device__ __forceinline__ bool reduce_last(double (&v)[ND], KrylovDev& kd, double* red) {
  __shared__ double ws[RT / 32][ND];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < ND; ++k) {
    double a = v[k];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) ws[w][k] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      double a = 0.0;
      for (int q = 0; q < RT / 32; ++q) a += ws[q][k];
      kd.part[blockIdx.x * ND + k] = a;
    }
    __threadfence();
    unsigned t = atomicAdd(kd.ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < ND; ++k) {
    double a = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += RT) a += __ldcg(&kd.part[b * ND + k]);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) ws[w][k] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      double a = 0.0;
      for (int q = 0; q < RT / 32; ++q) a += ws[q][k];
      red[k] = a;
    }
    *kd.ticket = 0u;
  }
  return true;
}

#define GRID_LOOP(i) for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT)

// ||a||^2 -> S[slot]
__global__ void __launch_bounds__(RT) k_norm2(const double* __restrict__ a, int64_t n, KrylovDev kd, int slot) {
  if (kr_skip(kd)) return;
  double v[1] = {0.0};
  GRID_LOOP(i) v[0] += a[i] * a[i];
  double red[1];
  if (reduce_last<1>(v, kd, red) && threadIdx.x == 0) kd.S[slot] = red[0];
}

// t = b - y, ||t||^2 -> S[slot]
__global__ void __launch_bounds__(RT) k_residual(const double* __restrict__ b, const double* __restrict__ y,
                                                 double* __restrict__ t, int64_t n, KrylovDev kd, int slot) {
  if (kr_skip(kd)) return;
  double v[1] = {0.0};
  GRID_LOOP(i) {
    double r = b[i] - y[i];
    t[i] = r;
    v[0] += r * r;
  }
  double red[1];
  if (reduce_last<1>(v, kd, red) && threadIdx.x == 0) kd.S[slot] = red[0];
}

// BiCG part, start of step j: (j == 0: rho0 = -omega rho0), rho1 = <r_j, rt>,
// beta = alpha rho1 / rho0, rho0 = rho1.
__global__ void __launch_bounds__(RT) k_bicg_rho(const double* __restrict__ rj, const double* __restrict__ rt,
                                                 int64_t n, KrylovDev kd, int j) {
  if (kr_skip(kd)) return;
  double v[1] = {0.0};
  GRID_LOOP(i) v[0] += rj[i] * rt[i];
  double red[1];
  if (reduce_last<1>(v, kd, red) && threadIdx.x == 0) {
    double* S = kd.S;
    if (j == 0) S[S_RHO0] = -S[S_OMEGA] * S[S_RHO0];
    double rho1 = red[0];
    if (S[S_RHO0] == 0.0) S[S_BREAK] = 1.0;
    S[S_BETA] = (S[S_RHO0] != 0.0) ? S[S_ALPHA] * rho1 / S[S_RHO0] : 0.0;
    S[S_RHO0] = rho1;
  }
}

// u_i = r_i - beta u_i, i = 0..j
__global__ void __launch_bounds__(RT) k_bicg_u(double* __restrict__ u0, double* __restrict__ u1,
                                               const double* __restrict__ r0, const double* __restrict__ r1,
                                               int64_t n, KrylovDev kd, int j) {
  if (kr_skip(kd)) return;
  const double beta = kd.S[S_BETA];
  GRID_LOOP(i) {
    u0[i] = r0[i] - beta * u0[i];
    if (j >= 1) u1[i] = r1[i] - beta * u1[i];
  }
}

// gamma = <u_{j+1}, rt>, alpha = rho0 / gamma
__global__ void __launch_bounds__(RT) k_bicg_gamma(const double* __restrict__ uj1, const double* __restrict__ rt,
                                                   int64_t n, KrylovDev kd) {
  if (kr_skip(kd)) return;
  double v[1] = {0.0};
  GRID_LOOP(i) v[0] += uj1[i] * rt[i];
  double red[1];
  if (reduce_last<1>(v, kd, red) && threadIdx.x == 0) {
    double* S = kd.S;
    double g = red[0];
    if (g == 0.0) S[S_BREAK] = 1.0;
    S[S_ALPHA] = (g != 0.0) ? S[S_RHO0] / g : 0.0;
  }
}

// r_i -= alpha u_{i+1} (i = 0..j), x += alpha u_0, ||r_0||^2 -> S[S_RN2]
__global__ void __launch_bounds__(RT) k_bicg_r(double* __restrict__ r0, double* __restrict__ r1,
                                               const double* __restrict__ u0, const double* __restrict__ u1,
                                               const double* __restrict__ u2, double* __restrict__ x,
                                               int64_t n, KrylovDev kd, int j) {
  if (kr_skip(kd)) return;
  const double alpha = kd.S[S_ALPHA];
  double v[1] = {0.0};
  GRID_LOOP(i) {
    double a = r0[i] - alpha * u1[i];
    r0[i] = a;
    if (j >= 1) r1[i] = r1[i] - alpha * u2[i];
    x[i] = x[i] + alpha * u0[i];
    v[0] += a * a;
  }
  double red[1];
  if (reduce_last<1>(v, kd, red) && threadIdx.x == 0) kd.S[S_RN2] = red[0];
}

// MR part (1): sigma1 = <r1,r1>, gamma'_1 = <r0,r1>/sigma1, tau12 = <r2,r1>/sigma1
__global__ void __launch_bounds__(RT) k_mr1(const double* __restrict__ r0, const double* __restrict__ r1,
                                            const double* __restrict__ r2, int64_t n, KrylovDev kd) {
  if (kr_skip(kd)) return;
  double v[3] = {0.0, 0.0, 0.0};
  GRID_LOOP(i) {
    double a = r1[i];
    v[0] += a * a;
    v[1] += r0[i] * a;
    v[2] += r2[i] * a;
  }
  double red[3];
  if (reduce_last<3>(v, kd, red) && threadIdx.x == 0) {
    double* S = kd.S;
    double s1 = red[0];
    if (s1 == 0.0) S[S_BREAK] = 1.0;
    S[S_SIGMA1] = s1;
    S[S_GP1] = (s1 != 0.0) ? red[1] / s1 : 0.0;
    S[S_TAU12] = (s1 != 0.0) ? red[2] / s1 : 0.0;
  }
}

// MR part (2): r2 -= tau12 r1; sigma2 = <r2,r2>; gamma'_2 = <r0,r2>/sigma2;
// gamma_2 = gamma'_2, omega = gamma_2, gamma_1 = gamma'_1 - tau12 gamma_2, gamma''_1 = gamma_2
__global__ void __launch_bounds__(RT) k_mr2(const double* __restrict__ r0, const double* __restrict__ r1,
                                            double* __restrict__ r2, int64_t n, KrylovDev kd) {
  if (kr_skip(kd)) return;
  const double tau = kd.S[S_TAU12];
  double v[2] = {0.0, 0.0};
  GRID_LOOP(i) {
    double a = r2[i] - tau * r1[i];
    r2[i] = a;
    v[0] += a * a;
    v[1] += r0[i] * a;
  }
  double red[2];
  if (reduce_last<2>(v, kd, red) && threadIdx.x == 0) {
    double* S = kd.S;
    double s2 = red[0];
    if (s2 == 0.0) S[S_BREAK] = 1.0;
    double gp2 = (s2 != 0.0) ? red[1] / s2 : 0.0;
    S[S_GP2] = gp2;
    S[S_G2] = gp2;
    S[S_OMEGA] = gp2;
    if (gp2 == 0.0) S[S_BREAK] = 1.0;
    S[S_G1] = S[S_GP1] - S[S_TAU12] * gp2;
    S[S_GPP1] = gp2;
  }
}

// MR part (3): x += g1 r0 + gpp1 r1; r0 -= gp2 r2 + gp1 r1; u0 -= g2 u2 + g1 u1; ||r0||^2
__global__ void __launch_bounds__(RT) k_mr3(double* __restrict__ x, double* __restrict__ r0,
                                            const double* __restrict__ r1, const double* __restrict__ r2,
                                            double* __restrict__ u0, const double* __restrict__ u1,
                                            const double* __restrict__ u2, int64_t n, KrylovDev kd) {
  if (kr_skip(kd)) return;
  const double* S = kd.S;
  const double g1 = S[S_G1], gpp1 = S[S_GPP1], gp2 = S[S_GP2], gp1 = S[S_GP1], g2 = S[S_G2];
  double v[1] = {0.0};
  GRID_LOOP(i) {
    double a0 = r0[i], a1 = r1[i];
    x[i] = x[i] + (g1 * a0 + gpp1 * a1);
    double nr = a0 - (gp2 * r2[i] + gp1 * a1);
    r0[i] = nr;
    u0[i] = u0[i] - (g2 * u2[i] + g1 * u1[i]);
    v[0] += nr * nr;
  }
  double red[1];
  if (reduce_last<1>(v, kd, red) && threadIdx.x == 0) kd.S[S_RN2] = red[0];
}

__global__ void k_exit_check(KrylovDev kd, double tol, double qoff) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int* f = kd.flags;
  double* S = kd.S;
  if (f[F_DONE]) return;
  f[F_REPLACE] = 0;
  if (S[S_BREAK] != 0.0) {
    f[F_DONE] = 1;
    f[F_STATUS] = SAP_ERR_BREAKDOWN;
    S[S_QUART] = S[S_IT] + qoff;
    return;
  }
  f[F_CHECK] = (sqrt(S[S_RN2]) <= tol * sqrt(S[S_BTN2])) ? 1 : 0;
}

__global__ void k_exit_decide(KrylovDev kd, double tol, double qoff) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int* f = kd.flags;
  double* S = kd.S;
  if (f[F_DONE]) return;
  if (f[F_CHECK]) {
    f[F_CHECK] = 0;
    const double rel = sqrt(S[S_TN2]) / sqrt(S[S_BN2]);
    S[S_RELRES] = rel;
    if (rel <= tol) {
      f[F_DONE] = 1;
      f[F_STATUS] = SAP_OK;
      S[S_QUART] = S[S_IT] + qoff;
      return;
    }
    // a failed confirmation after the MR update restarts the method from x
    // (r^0 = M^{-1}(b - A x), then k_restart); after matvec 1 or 3 the
    // iteration goes on unchanged
    if (qoff == 1.0) {
      f[F_REPLACE] = 1;
      f[F_RESTARTS] += 1;
    }
  }
  if (qoff == 1.0) S[S_IT] += 1.0;
}

// Restart after a residual replacement: shadow residual r~0 = r^0, u^0 = 0,
// rho0 = 1, alpha = 0, omega = 1 (the state of a fresh start); gated on F_REPLACE.
__global__ void k_restart(const double* __restrict__ r0, double* __restrict__ rt, double* __restrict__ u0,
                          int64_t n, KrylovDev kd) {
  if (kr_skip(kd)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    rt[i] = r0[i];
    u0[i] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    kd.S[S_RHO0] = 1.0;
    kd.S[S_ALPHA] = 0.0;
    kd.S[S_OMEGA] = 1.0;
  }
}

__global__ void k_init_scalars(double* S) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    for (int k = 0; k < S_COUNT; ++k) S[k] = 0.0;
    S[S_RHO0] = 1.0;
    S[S_ALPHA] = 0.0;
    S[S_OMEGA] = 1.0;
  }
}

// ---- preconditioned conjugate gradient (Sec. 3: the outer iteration for a
// symmetric positive definite A; Saad 2003, Algorithm 9.1) ----
// Every kernel carries the gate of its KrylovDev (see GateMode).
// p = z and (r, z) -> S[S_RHO0]: the start (and a restart) of the iteration
__global__ void __launch_bounds__(RT) k_cg_start(const double* __restrict__ r, const double* __restrict__ z,
                                                 double* __restrict__ p, int64_t n, KrylovDev kd) {
  if (kr_skip(kd)) return;
  double v[1] = {0.0};
  GRID_LOOP(i) {
    const double zi = z[i];
    p[i] = zi;
    v[0] += r[i] * zi;
  }
  double red[1];
  if (reduce_last<1>(v, kd, red) && threadIdx.x == 0) kd.S[S_RHO0] = red[0];
}

// alpha = (r, z) / (p, A p) -> S[S_ALPHA]; (p, A p) = 0 flags a breakdown
__global__ void __launch_bounds__(RT) k_cg_alpha(const double* __restrict__ p, const double* __restrict__ q,
                                                 int64_t n, KrylovDev kd) {
  if (kr_skip(kd)) return;
  double v[1] = {0.0};
  GRID_LOOP(i) v[0] += p[i] * q[i];
  double red[1];
  if (reduce_last<1>(v, kd, red) && threadIdx.x == 0) {
    double* S = kd.S;
    if (red[0] == 0.0) {
      S[S_BREAK] = 1.0;
      S[S_ALPHA] = 0.0;
    } else {
      S[S_ALPHA] = S[S_RHO0] / red[0];
    }
  }
}

// x += alpha p, r -= alpha A p, ||r||^2 -> S[S_RN2]
__global__ void __launch_bounds__(RT) k_cg_xr(double* __restrict__ x, double* __restrict__ r,
                                              const double* __restrict__ p, const double* __restrict__ q, int64_t n,
                                              KrylovDev kd) {
  if (kr_skip(kd)) return;
  const double a = kd.S[S_ALPHA];
  double v[1] = {0.0};
  GRID_LOOP(i) {
    x[i] += a * p[i];
    const double ri = r[i] - a * q[i];
    r[i] = ri;
    v[0] += ri * ri;
  }
  double red[1];
  if (reduce_last<1>(v, kd, red) && threadIdx.x == 0) kd.S[S_RN2] = red[0];
}

// beta = (r, z) / (r, z)_previous -> S[S_BETA], the new (r, z) -> S[S_RHO0];
// a zero previous (r, z) flags a breakdown
__global__ void __launch_bounds__(RT) k_cg_beta(const double* __restrict__ r, const double* __restrict__ z,
                                                int64_t n, KrylovDev kd) {
  if (kr_skip(kd)) return;
  double v[1] = {0.0};
  GRID_LOOP(i) v[0] += r[i] * z[i];
  double red[1];
  if (reduce_last<1>(v, kd, red) && threadIdx.x == 0) {
    double* S = kd.S;
    if (S[S_RHO0] == 0.0) {
      S[S_BREAK] = 1.0;
      S[S_BETA] = 0.0;
    } else {
      S[S_BETA] = red[0] / S[S_RHO0];
    }
    S[S_RHO0] = red[0];
  }
}

// p = z + beta p
__global__ void __launch_bounds__(RT) k_cg_p(const double* __restrict__ z, double* __restrict__ p, int64_t n,
                                             KrylovDev kd) {
  if (kr_skip(kd)) return;
  const double bt = kd.S[S_BETA];
  GRID_LOOP(i) p[i] = z[i] + bt * p[i];
}

// dst = src (the restart's r = b - A x)
__global__ void __launch_bounds__(RT) k_copy_gated(const double* __restrict__ src, double* __restrict__ dst,
                                                   int64_t n, KrylovDev kd) {
  if (kr_skip(kd)) return;
  GRID_LOOP(i) dst[i] = src[i];
}

// CG exit test, first half (after x += alpha p, r -= alpha A p): unless
// finished, a breakdown finishes the solve, else flag a true-residual check
// when the recursive residual satisfies ||r|| <= tol ||b||.
__global__ void k_cg_check(KrylovDev kd, double tol) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int* f = kd.flags;
  double* S = kd.S;
  if (f[F_DONE]) return;
  f[F_REPLACE] = 0;
  if (S[S_BREAK] != 0.0) {
    f[F_DONE] = 1;
    f[F_STATUS] = SAP_ERR_BREAKDOWN;
    S[S_QUART] = S[S_IT] + 1.0;
    return;
  }
  f[F_CHECK] = (sqrt(S[S_RN2]) <= tol * sqrt(S[S_BN2])) ? 1 : 0;
}

// Second half, after the gated true residual: the step is complete; accept,
// or flag the restart from x (r = b - A x, z = M^{-1} r, p = z) when the
// confirmation failed; the iteration cap finishes the solve.
__global__ void k_cg_decide(KrylovDev kd, double tol, int max_iters) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int* f = kd.flags;
  double* S = kd.S;
  if (f[F_DONE]) return;
  S[S_IT] += 1.0;
  if (f[F_CHECK]) {
    f[F_CHECK] = 0;
    const double rel = sqrt(S[S_TN2]) / sqrt(S[S_BN2]);
    S[S_RELRES] = rel;
    if (rel <= tol) {
      f[F_DONE] = 1;
      f[F_STATUS] = SAP_OK;
      S[S_QUART] = S[S_IT];
      return;
    }
    f[F_REPLACE] = 1;
    f[F_RESTARTS] += 1;
  }
  if (S[S_IT] >= (double)max_iters) {
    f[F_DONE] = 1;
    f[F_STATUS] = SAP_ERR_NOT_CONVERGED;
    S[S_QUART] = S[S_IT];
  }
}

}  // namespace

int krylov_grid(int64_t n) {
  int64_t g = (n + RT - 1) / RT;
  if (g > kKrylovBlocks) g = kKrylovBlocks;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t kr_init(KrylovDev kd, cudaStream_t s) {
  count_launches(1);
  k_init_scalars<<<1, 32, 0, s>>>(kd.S);
  return cudaGetLastError();
}
cudaError_t kr_exit_check(KrylovDev kd, double tol, double qoff, cudaStream_t s) {
  count_launches(1);
  k_exit_check<<<1, 32, 0, s>>>(kd, tol, qoff);
  return cudaGetLastError();
}
cudaError_t kr_restart(const double* r0, double* rt, double* u0, int64_t n, KrylovDev kd, cudaStream_t s) {
  count_launches(1);
  k_restart<<<krylov_grid(n), RT, 0, s>>>(r0, rt, u0, n, kd);
  return cudaGetLastError();
}
__global__ void k_while_next(cudaGraphConditionalHandle hnd, int* flags, int step, int cap) {
  const int c = flags[F_ROUNDS] + step;
  flags[F_ROUNDS] = c;
  cudaGraphSetConditional(hnd, (flags[F_DONE] == 0 && c < cap) ? 1u : 0u);
}

cudaError_t kr_while_next(cudaGraphConditionalHandle hnd, int* flags, int step, int cap, cudaStream_t s) {
  count_launches(1);
  k_while_next<<<1, 1, 0, s>>>(hnd, flags, step, cap);
  return cudaGetLastError();
}

cudaError_t kr_exit_decide(KrylovDev kd, double tol, double qoff, cudaStream_t s) {
  count_launches(1);
  k_exit_decide<<<1, 32, 0, s>>>(kd, tol, qoff);
  return cudaGetLastError();
}
cudaError_t kr_norm2(const double* a, int64_t n, KrylovDev kd, int slot, cudaStream_t s) {
  count_launches(1);
  k_norm2<<<krylov_grid(n), RT, 0, s>>>(a, n, kd, slot);
  return cudaGetLastError();
}
cudaError_t kr_residual(const double* b, const double* y, double* t, int64_t n, KrylovDev kd, int slot,
                        cudaStream_t s) {
  count_launches(1);
  k_residual<<<krylov_grid(n), RT, 0, s>>>(b, y, t, n, kd, slot);
  return cudaGetLastError();
}
cudaError_t kr_bicg_rho(const double* rj, const double* rt, int64_t n, KrylovDev kd, int j, cudaStream_t s) {
  count_launches(1);
  k_bicg_rho<<<krylov_grid(n), RT, 0, s>>>(rj, rt, n, kd, j);
  return cudaGetLastError();
}
cudaError_t kr_bicg_u(double* u0, double* u1, const double* r0, const double* r1, int64_t n, KrylovDev kd, int j,
                      cudaStream_t s) {
  count_launches(1);
  k_bicg_u<<<krylov_grid(n), RT, 0, s>>>(u0, u1, r0, r1, n, kd, j);
  return cudaGetLastError();
}
cudaError_t kr_bicg_gamma(const double* uj1, const double* rt, int64_t n, KrylovDev kd, cudaStream_t s) {
  count_launches(1);
  k_bicg_gamma<<<krylov_grid(n), RT, 0, s>>>(uj1, rt, n, kd);
  return cudaGetLastError();
}
cudaError_t kr_bicg_r(double* r0, double* r1, const double* u0, const double* u1, const double* u2, double* x,
                      int64_t n, KrylovDev kd, int j, cudaStream_t s) {
  count_launches(1);
  k_bicg_r<<<krylov_grid(n), RT, 0, s>>>(r0, r1, u0, u1, u2, x, n, kd, j);
  return cudaGetLastError();
}
cudaError_t kr_mr(double* x, double* r0, double* r1, double* r2, double* u0, const double* u1, const double* u2,
                  int64_t n, KrylovDev kd, cudaStream_t s) {
  int g = krylov_grid(n);
  count_launches(1);
  k_mr1<<<g, RT, 0, s>>>(r0, r1, r2, n, kd);
  count_launches(1);
  k_mr2<<<g, RT, 0, s>>>(r0, r1, r2, n, kd);
  count_launches(1);
  k_mr3<<<g, RT, 0, s>>>(x, r0, r1, r2, u0, u1, u2, n, kd);
  return cudaGetLastError();
}

// ---- failure-detection self-test ----
// One thread waits, with the bounded mbarrier wait of the library's kernels,
// on a barrier whose phase nothing completes (no arrival, no copy in flight);
// after `limit` polls the wait records the timeout in *err and the kernel
// ends normally, leaving the context usable.
__global__ void k_wait_selftest(int limit, int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
  }
  __syncthreads();
  bool failed = false;
  if (threadIdx.x == 0) tc::mbar_wait_bounded(&bar, 0u, limit, err, failed);
}

cudaError_t launch_wait_selftest(int limit, int* err, cudaStream_t s) {
  count_launches(1);
  k_wait_selftest<<<1, 32, 0, s>>>(limit, err);
  return cudaGetLastError();
}

cudaError_t kr_cg_start(const double* r, const double* z, double* p, int64_t n, KrylovDev kd, cudaStream_t s) {
  count_launches(1);
  k_cg_start<<<krylov_grid(n), RT, 0, s>>>(r, z, p, n, kd);
  return cudaGetLastError();
}
cudaError_t kr_cg_alpha(const double* p, const double* q, int64_t n, KrylovDev kd, cudaStream_t s) {
  count_launches(1);
  k_cg_alpha<<<krylov_grid(n), RT, 0, s>>>(p, q, n, kd);
  return cudaGetLastError();
}
cudaError_t kr_cg_xr(double* x, double* r, const double* p, const double* q, int64_t n, KrylovDev kd,
                     cudaStream_t s) {
  count_launches(1);
  k_cg_xr<<<krylov_grid(n), RT, 0, s>>>(x, r, p, q, n, kd);
  return cudaGetLastError();
}
cudaError_t kr_cg_beta(const double* r, const double* z, int64_t n, KrylovDev kd, cudaStream_t s) {
  count_launches(1);
  k_cg_beta<<<krylov_grid(n), RT, 0, s>>>(r, z, n, kd);
  return cudaGetLastError();
}
cudaError_t kr_cg_p(const double* z, double* p, int64_t n, KrylovDev kd, cudaStream_t s) {
  count_launches(1);
  k_cg_p<<<krylov_grid(n), RT, 0, s>>>(z, p, n, kd);
  return cudaGetLastError();
}
cudaError_t kr_copy(const double* src, double* dst, int64_t n, KrylovDev kd, cudaStream_t s) {
  count_launches(1);
  k_copy_gated<<<krylov_grid(n), RT, 0, s>>>(src, dst, n, kd);
  return cudaGetLastError();
}
cudaError_t kr_cg_check(KrylovDev kd, double tol, cudaStream_t s) {
  count_launches(1);
  k_cg_check<<<1, 32, 0, s>>>(kd, tol);
  return cudaGetLastError();
}
cudaError_t kr_cg_decide(KrylovDev kd, double tol, int max_iters, cudaStream_t s) {
  count_launches(1);
  k_cg_decide<<<1, 32, 0, s>>>(kd, tol, max_iters);
  return cudaGetLastError();
}

}  // namespace sap
