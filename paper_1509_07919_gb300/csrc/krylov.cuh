// Device scalars and launchers of the fused BiCGStab(2) vector kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "sap_internal.cuh"

namespace sap {

// Slots of the device scalar array of one Krylov solve.
enum ScalarSlot {
  S_RHO0 = 0, S_ALPHA, S_OMEGA, S_BETA, S_SIGMA1, S_GP1, S_TAU12, S_GP2, S_G1, S_G2, S_GPP1,
  S_RN2,      // ||r^0||^2 after the last update
  S_BN2,      // ||b||^2
  S_BTN2,     // ||M^{-1} b||^2
  S_TN2,      // ||b - A x||^2 (true residual)
  S_BREAK,    // breakdown flag (nonzero)
  S_IT,       // completed outer iterations
  S_QUART,    // iterations (in quarters) at the accepted exit
  S_RELRES,   // true relative residual of the last check
  S_COUNT
};

constexpr int kKrylovBlocks = 2 * 152;  // fixed reduction grid (two CTAs per SM)

struct KrylovDev {
  double* S;           // S_COUNT scalars
  double* part;        // kKrylovBlocks * 4 partial sums
  unsigned* ticket;    // last-block counter (returns to 0 after each reduction)
  int* flags = nullptr;   // F_COUNT control flags of the device-driven iteration
  int gmode = 0;          // GateMode of the launch carrying this struct
};

int krylov_grid(int64_t n);
cudaError_t kr_init(KrylovDev kd, cudaStream_t s);
cudaError_t kr_norm2(const double* a, int64_t n, KrylovDev kd, int slot, cudaStream_t s);
cudaError_t kr_residual(const double* b, const double* y, double* t, int64_t n, KrylovDev kd, int slot,
                        cudaStream_t s);
cudaError_t kr_bicg_rho(const double* rj, const double* rt, int64_t n, KrylovDev kd, int j, cudaStream_t s);
cudaError_t kr_bicg_u(double* u0, double* u1, const double* r0, const double* r1, int64_t n, KrylovDev kd, int j,
                      cudaStream_t s);
cudaError_t kr_bicg_gamma(const double* uj1, const double* rt, int64_t n, KrylovDev kd, cudaStream_t s);
cudaError_t kr_bicg_r(double* r0, double* r1, const double* u0, const double* u1, const double* u2, double* x,
                      int64_t n, KrylovDev kd, int j, cudaStream_t s);
cudaError_t kr_mr(double* x, double* r0, double* r1, double* r2, double* u0, const double* u1, const double* u2,
                  int64_t n, KrylovDev kd, cudaStream_t s);
// Exit test at iteration S_IT + qoff, first half: unless finished, flag a true-
// residual check when ||r^0|| <= tol ||M^{-1} b|| (breakdown finishes the solve).
cudaError_t kr_exit_check(KrylovDev kd, double tol, double qoff, cudaStream_t s);
// Second half, after the gated true residual: accept (finish) or flag the
// residual replacement; qoff == 1 also completes the outer iteration.
cudaError_t kr_exit_decide(KrylovDev kd, double tol, double qoff, cudaStream_t s);
// End of one round of the device-driven loop: flags[F_ROUNDS] += step, and
// the loop's WHILE condition set to continue while the solve is not done and
// the count is below cap.
cudaError_t kr_while_next(cudaGraphConditionalHandle hnd, int* flags, int step, int cap, cudaStream_t s);
// Preconditioned CG (Saad, Alg. 9.1), each launch gated by kd.gmode: p = z
// with (r, z) -> S_RHO0; alpha = S_RHO0 / (p, q); x += alpha p, r -= alpha q
// with ||r||^2 -> S_RN2; beta = (r, z) / S_RHO0 (S_RHO0 updated);
// p = z + beta p.  A zero denominator sets S_BREAK.  Exit test in two halves
// around the gated true residual (kr_cg_check, kr_cg_decide: whole steps,
// restart flag on a failed confirmation, the iteration cap on the device);
// kr_copy: dst = src, gated.
cudaError_t kr_cg_start(const double* r, const double* z, double* p, int64_t n, KrylovDev kd, cudaStream_t s);
cudaError_t kr_cg_alpha(const double* p, const double* q, int64_t n, KrylovDev kd, cudaStream_t s);
cudaError_t kr_cg_xr(double* x, double* r, const double* p, const double* q, int64_t n, KrylovDev kd,
                     cudaStream_t s);
cudaError_t kr_cg_beta(const double* r, const double* z, int64_t n, KrylovDev kd, cudaStream_t s);
cudaError_t kr_cg_p(const double* z, double* p, int64_t n, KrylovDev kd, cudaStream_t s);
cudaError_t kr_copy(const double* src, double* dst, int64_t n, KrylovDev kd, cudaStream_t s);
cudaError_t kr_cg_check(KrylovDev kd, double tol, cudaStream_t s);
cudaError_t kr_cg_decide(KrylovDev kd, double tol, int max_iters, cudaStream_t s);
// restart after a residual replacement (gated on the replacement flag)
cudaError_t kr_restart(const double* r0, double* rt, double* u0, int64_t n, KrylovDev kd, cudaStream_t s);

}  // namespace sap
