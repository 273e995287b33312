// Part III: BPDN (Eq. 7, Dirac basis, real image) by Douglas-Rachford splitting
// (Section 2.3), with the projection onto the data-fidelity ball computed by
// dual forward-backward:
//
//   z_0 = Re Phi^H y,   gamma = gamma_frac * max|z_0|,   u = 0
//   repeat T times:
//     repeat K times:  x = z - Re Phi^H u
//                      d = u/mu + Phi x - y
//                      u = max(0, 1 - eps/||d||) mu d
//     x = z - Re Phi^H u                       (x = P_B(z))
//     z = z + lambda (soft(2x - z, gamma) - x)
//   return x
//
// All norms are FP64 reductions with a fixed order; the ball-projection scale is
// computed on the device, so an iteration needs no host round trip.
#include "plan.h"

namespace wproj {

namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 304;   // 2 x 152 SMs

// d = u/mu + r - y (written over r); partial sums of |d|^2
__global__ void __launch_bounds__(kRedThreads)
k_dual_residual(int64_t m, const float2 *__restrict__ u, float2 *__restrict__ r,
                const float2 *__restrict__ y, float inv_mu, double *__restrict__ part) {
  double acc = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x) {
    const float2 uu = u[i], rr = r[i], yy = y[i];
    const float2 d = make_float2(uu.x * inv_mu + rr.x - yy.x, uu.y * inv_mu + rr.y - yy.y);
    r[i] = d;
    acc += double(d.x) * d.x + double(d.y) * d.y;
  }
  const double t = block_sum_d<kRedThreads>(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// scal[0] = max(0, 1 - eps/||d||) * mu
__global__ void k_ball_scale(const double *__restrict__ part, int n, double eps, double mu,
                             double *__restrict__ scal) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0;
  for (int i = 0; i < n; ++i) s += part[i];
  const double nd = sqrt(s);
  const double f = (nd > 0) ? fmax(0.0, 1.0 - eps / nd) : 0.0;
  scal[0] = f * mu;
  scal[1] = nd;
}

__global__ void k_dual_update(int64_t m, const float2 *__restrict__ d, const double *__restrict__ scal,
                              float2 *__restrict__ u) {
  const float f = float(scal[0]);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x)
    u[i] = cscale(d[i], f);
}

// z = z + lambda (soft(2x - z, gamma) - x), gamma = scal[2]
__global__ void k_dr_update(int64_t n, const float *__restrict__ x, float *__restrict__ z, float lambda,
                            const double *__restrict__ scal) {
  const float gamma = float(scal[2]);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float xi = x[i], zi = z[i];
    const float a = 2.f * xi - zi;
    const float sa = copysignf(fmaxf(fabsf(a) - gamma, 0.f), a);
    z[i] = zi + lambda * (sa - xi);
  }
}

__global__ void __launch_bounds__(kRedThreads)
k_absmax_part(int64_t n, const float *__restrict__ x, double *__restrict__ part) {
  float mx = 0.f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    mx = fmaxf(mx, fabsf(x[i]));
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ float red[kRedThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < kRedThreads / 32; ++i) t = fmaxf(t, red[i]);
    part[blockIdx.x] = t;
  }
}

// scal[2] = frac * max(part)
__global__ void k_gamma(const double *__restrict__ part, int n, double frac, double *__restrict__ scal) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double mx = 0;
  for (int i = 0; i < n; ++i) mx = fmax(mx, part[i]);
  scal[2] = frac * mx;
}

template <int ABS>
__global__ void __launch_bounds__(kRedThreads)
k_sum_part(int64_t n, const float *__restrict__ x, double *__restrict__ part) {
  double acc = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double v = x[i];
    acc += ABS ? fabs(v) : v * v;
  }
  const double t = block_sum_d<kRedThreads>(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kRedThreads)
k_resid_part(int64_t m, const float2 *__restrict__ a, const float2 *__restrict__ b, double *__restrict__ part) {
  double acc = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x) {
    const double dx = double(a[i].x) - b[i].x, dy = double(a[i].y) - b[i].y;
    acc += dx * dx + dy * dy;
  }
  const double t = block_sum_d<kRedThreads>(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_sum_parts(const double *__restrict__ part, int n, double *__restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0;
  for (int i = 0; i < n; ++i) s += part[i];
  *out = s;
}

// x = z / sqrt(scal[3])
__global__ void k_normalise(int64_t n, const float *__restrict__ z, const double *__restrict__ scal,
                            float *__restrict__ x) {
  const float f = float(1.0 / sqrt(scal[3]));
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] = z[i] * f;
}

// the unit impulse at flat index `at`
__global__ void k_impulse(int64_t n, float *__restrict__ x, int64_t at) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] = i == at ? 1.f : 0.f;
}

int grid_for(int64_t n) { return (int)std::min<int64_t>(kRedBlocks, std::max<int64_t>(1, ceil_div(n, kRedThreads))); }

wproj_status ensure_solver_buffers(wproj_plan *p) {
  const int64_t n = int64_t(p->g.N) * p->g.N;
  WPROJ_TRY(p->s_z.ensure(sizeof(float) * n));
  WPROJ_TRY(p->s_x.ensure(sizeof(float) * n));
  WPROJ_TRY(p->s_u.ensure(sizeof(float2) * std::max<int64_t>(1, p->m)));
  WPROJ_TRY(p->s_r.ensure(sizeof(float2) * std::max<int64_t>(1, p->m)));
  WPROJ_TRY(p->s_scal.ensure(sizeof(double) * (8 + kRedBlocks)));
  return WPROJ_OK;
}

}  // namespace

// ||Phi||^2 by power iteration on Re Phi^H Phi from the unit impulse at the image
// centre (flat spectrum: no row of Phi is orthogonal to it).
wproj_status power_norm2_impl(wproj_plan *p, int iters, double *out, cudaStream_t s) {
  WPROJ_TRY(ensure_solver_buffers(p));
  const int64_t n = int64_t(p->g.N) * p->g.N;
  // scratch only: the Douglas-Rachford state (z, u, gamma) is left untouched
  float *x = p->xtmp.as<float>(), *z = p->s_x.as<float>();
  float2 *r = p->s_r.as<float2>();
  double *scal = p->s_scal.as<double>();
  double *part = scal + 8;
  k_impulse<<<grid_for(n), kRedThreads, 0, s>>>(n, x, int64_t(p->g.N / 2) * p->g.N + p->g.N / 2);
  WPROJ_CHECK_LAUNCH("power iteration start");
  p->launches += 1;
  for (int it = 0; it < iters; ++it) {
    WPROJ_TRY(apply_phi(p, x, nullptr, r, s));
    WPROJ_TRY(apply_phi_adj(p, r, z, nullptr, nullptr, 0, s));
    const int nb = grid_for(n);
    k_sum_part<0><<<nb, kRedThreads, 0, s>>>(n, z, part);
    k_sum_parts<<<1, 1, 0, s>>>(part, nb, scal + 3);
    k_normalise<<<grid_for(n), kRedThreads, 0, s>>>(n, z, scal, x);
    WPROJ_CHECK_LAUNCH("power iteration");
    p->launches += 3;
  }
  double h = 0;
  WPROJ_CUDA(cudaMemcpyAsync(&h, scal + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  *out = sqrt(h);
  return WPROJ_OK;
}

wproj_status solve_bpdn_impl(wproj_plan *p, const float2 *y, double eps, const wproj_dr_params &prm,
                             float *x_out, wproj_solve_info *info, cudaStream_t s) {
  const bool resume = prm.resume && p->dr_valid;
  if (!resume) WPROJ_TRY(ensure_solver_buffers(p));
  double phi_norm2 = prm.phi_norm2;
  if (!(phi_norm2 > 0) && resume) phi_norm2 = p->dr_phi_norm2;
  if (!(phi_norm2 > 0)) WPROJ_TRY(power_norm2_impl(p, prm.power_iters, &phi_norm2, s));
  if (!(phi_norm2 > 0) || !isfinite(phi_norm2))
    return fail(WPROJ_ERR_INVALID_ARG, "solve_bpdn: ||Phi||^2 is zero or not finite");
  const double mu = 1.0 / phi_norm2;
  const int64_t n = int64_t(p->g.N) * p->g.N;
  const int64_t m = p->m;
  // Psi (Eq. 7): 0 = Dirac; else Daubechies-psi wavelets, orthonormal, so the
  // projection onto the constraint set in coefficient space is Psi^T P(Psi z) with
  // P the image-space projection: z, the soft threshold and the DR update live
  // in coefficient space; the inner loop runs on the image zi = Psi z.
  const int psi = prm.psi, lev = prm.psi_levels, N = p->g.N;
  if (psi) {
    WPROJ_TRY(p->s_zi.ensure(sizeof(float) * n));
    WPROJ_TRY(p->s_alpha.ensure(sizeof(float) * n));
    WPROJ_TRY(p->s_wwork.ensure(sizeof(float) * (n / 2 + 1)));
  }
  float *z = p->s_z.as<float>(), *x = p->s_x.as<float>();
  float *zi = psi ? p->s_zi.as<float>() : z;         // the image the projection starts from
  float *alpha = psi ? p->s_alpha.as<float>() : x;   // P(z) in the basis of z
  float *wk = p->s_wwork.as<float>();
  float2 *u = p->s_u.as<float2>(), *r = p->s_r.as<float2>();
  double *scal = p->s_scal.as<double>();
  double *part = scal + 8;
  const int nbm = grid_for(m), nbn = grid_for(n);

  if (!resume) {
    // z0 = Psi^T Re Phi^H y, gamma
    if (psi) {
      WPROJ_TRY(apply_phi_adj(p, y, x, nullptr, nullptr, 0, s));
      WPROJ_TRY(dwt2_impl(N, lev, psi, x, z, wk, &p->launches, s));
    } else {
      WPROJ_TRY(apply_phi_adj(p, y, z, nullptr, nullptr, 0, s));
    }
    ScopedTimer t(p, TC_SOLVER, s);
    k_absmax_part<<<nbn, kRedThreads, 0, s>>>(n, z, part);
    k_gamma<<<1, 1, 0, s>>>(part, nbn, prm.gamma_frac, scal);
    WPROJ_CUDA(cudaMemsetAsync(u, 0, sizeof(float2) * m, s));
    WPROJ_CHECK_LAUNCH("dr init");
    p->launches += 2;
  }
  p->dr_valid = true;
  p->dr_phi_norm2 = phi_norm2;
  for (int t_ = 0; t_ < prm.iters; ++t_) {
    if (psi) WPROJ_TRY(idwt2_impl(N, lev, psi, z, zi, wk, &p->launches, s));
    for (int j = 0; j < prm.inner_iters; ++j) {
      WPROJ_TRY(apply_phi_adj(p, u, x, nullptr, zi, 1, s));   // x = zi - Re Phi^H u
      WPROJ_TRY(apply_phi(p, x, nullptr, r, s));               // r = Phi x
      ScopedTimer t(p, TC_SOLVER, s);
      k_dual_residual<<<nbm, kRedThreads, 0, s>>>(m, u, r, y, float(1.0 / mu), part);
      k_ball_scale<<<1, 1, 0, s>>>(part, nbm, eps, mu, scal);
      k_dual_update<<<nbm, kRedThreads, 0, s>>>(m, r, scal, u);
      WPROJ_CHECK_LAUNCH("dual step");
      p->launches += 3;
    }
    WPROJ_TRY(apply_phi_adj(p, u, x, nullptr, zi, 1, s));     // x = P_B(zi)
    if (psi) WPROJ_TRY(dwt2_impl(N, lev, psi, x, alpha, wk, &p->launches, s));
    ScopedTimer t(p, TC_SOLVER, s);
    k_dr_update<<<nbn, kRedThreads, 0, s>>>(n, alpha, z, float(prm.lambda), scal);
    WPROJ_CHECK_LAUNCH("dr update");
    p->launches += 1;
  }
  if (prm.iters == 0) {
    if (psi) WPROJ_TRY(idwt2_impl(N, lev, psi, z, x, wk, &p->launches, s));
    else WPROJ_CUDA(cudaMemcpyAsync(x, z, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
  }
  WPROJ_CUDA(cudaMemcpyAsync(x_out, x, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
  if (info) {
    // residual ||y - Phi x|| and ||x||_1
    WPROJ_TRY(apply_phi(p, x, nullptr, r, s));
    k_resid_part<<<nbm, kRedThreads, 0, s>>>(m, r, y, part);
    k_sum_parts<<<1, 1, 0, s>>>(part, nbm, scal + 4);
    if (psi) WPROJ_TRY(dwt2_impl(N, lev, psi, x, alpha, wk, &p->launches, s));
    k_sum_part<1><<<nbn, kRedThreads, 0, s>>>(n, alpha, part);
    k_sum_parts<<<1, 1, 0, s>>>(part, nbn, scal + 5);
    WPROJ_CHECK_LAUNCH("solve info");
    double h[4];   // gamma, ||d||, ||y - Phi x||^2, ||x||_1
    WPROJ_CUDA(cudaMemcpyAsync(h, scal + 2, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
    WPROJ_CUDA(cudaStreamSynchronize(s));
    info->iters_done = prm.iters;
    info->phi_norm2 = phi_norm2;
    info->gamma = h[0];
    info->final_resid = sqrt(h[2]);
    info->final_l1 = h[3];
  }
  return WPROJ_OK;
}

wproj_status dr_state_get(wproj_plan *p, float *z, void *u, double *gamma, double *phi_norm2, cudaStream_t s) {
  if (!p->dr_valid) return fail(WPROJ_ERR_NOT_BUILT, "no Douglas-Rachford state (run a solve first)");
  const int64_t n = int64_t(p->g.N) * p->g.N;
  if (z) WPROJ_CUDA(cudaMemcpyAsync(z, p->s_z.ptr, sizeof(float) * n, cudaMemcpyDefault, s));
  if (u) WPROJ_CUDA(cudaMemcpyAsync(u, p->s_u.ptr, sizeof(float2) * p->m, cudaMemcpyDefault, s));
  double g = 0;
  WPROJ_CUDA(cudaMemcpyAsync(&g, p->s_scal.as<double>() + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  if (gamma) *gamma = g;
  if (phi_norm2) *phi_norm2 = p->dr_phi_norm2;
  return WPROJ_OK;
}

wproj_status dr_state_set(wproj_plan *p, const float *z, const void *u, double gamma, double phi_norm2,
                          cudaStream_t s) {
  WPROJ_TRY(ensure_solver_buffers(p));
  const int64_t n = int64_t(p->g.N) * p->g.N;
  WPROJ_CUDA(cudaMemcpyAsync(p->s_z.ptr, z, sizeof(float) * n, cudaMemcpyDefault, s));
  WPROJ_CUDA(cudaMemcpyAsync(p->s_u.ptr, u, sizeof(float2) * p->m, cudaMemcpyDefault, s));
  WPROJ_CUDA(cudaMemcpyAsync(p->s_scal.as<double>() + 2, &gamma, sizeof(double), cudaMemcpyHostToDevice, s));
  WPROJ_CUDA(cudaStreamSynchronize(s));
  p->dr_valid = true;
  p->dr_phi_norm2 = phi_norm2;
  return WPROJ_OK;
}

}  // namespace wproj
