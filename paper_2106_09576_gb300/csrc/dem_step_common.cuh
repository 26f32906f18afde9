// dem_step_common.cuh -- contact law, wall geometry and bookkeeping shared by the two
// step kernels (FP64: dem_step_fp64.cu, mixed precision: dem_step_mixed.cu).
//
// Both kernels evaluate every touching contact from each partner's side (full list), so
// no force is ever scattered to another particle: the sums need no atomics and are
// deterministic.  After the forces they integrate with velocity Verlet:
//   v^n       = v^{n-1/2} + a^n dt/2     (Eq. newvv)
//   v^{n+1/2} = v^n + a^n dt/2           (Eq. halfstep, next step)
//   x^{n+1}   = x^n + v^{n+1/2} dt
// and flag a contact search when |x^{n+1} - x_ref| > skin/2 (dynamic mode, Sec. 3.1).
#pragma once
#include "dem_device.cuh"

namespace demgb {

// ------------------------------------------------------------------ FP64 contact law
// Mirrors, operation by operation, the serial CPU statement of Eqs. normal_force,
// tangential_force, nonlinearkn..nonlinearetat, coulomb_overlap..coulomb_overlap3,
// torque_t and the constant rolling model.
__device__ __forceinline__ double dot3d(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
__device__ __forceinline__ void cross3d(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// Linear model (Eqs. linearkn, linearetan): k and eta from the pair's R_e, m_e, Y_e and
// the characteristic impact velocity V; the same constants act tangentially.
__device__ __forceinline__ void linear_constants_d(double Re, double me, double Ye, double V, double lin_den,
                                                   double* k, double* eta) {
  const double sR = sqrt(Re);
  const double arg = 15.0 * me * V * V / (16.0 * sR * Ye);
  *k = 16.0 / 15.0 * sR * Ye * pow(arg, 0.2);
  *eta = sqrt(4.0 * me * (*k) / lin_den);
}

// vom: V_omega of the viscous rolling model ((R_i w_i + R_j w_j) x n, or R_i (w_i - Omega)
// x n against a wall); lin: linear model constants {V, 1 + (pi/ln e)^2} or null.
__device__ __forceinline__ void law_d(const double* nrm, double dn, const double* vij, const double* dw,
                                      const double* vom, double Re, double me, double Ye, double Ge,
                                      double ceta, double mu, double mur, int rolling, const double* lin,
                                      double dt, double* H, bool incr, double* Fsum, double* nxFt,
                                      double* Mr) {
  double vn = dot3d(vij, nrm);
  double vrn[3], vrt[3];
  for (int d = 0; d < 3; d++) {
    vrn[d] = vn * nrm[d];
    vrt[d] = vij[d] - vrn[d];
  }
  if (incr)
    for (int d = 0; d < 3; d++) H[d] = H[d] + vrt[d] * dt;
  double kn, kt, eta_n, eta_t;
  if (lin == nullptr) {
    double sq = sqrt(Re * dn);
    kn = 4.0 / 3.0 * Ye * sq;
    double Sn = 2.0 * Ye * sq;
    kt = 8.0 * Ge * sq;
    double St = 8.0 * Ge * sq;
    eta_n = ceta * sqrt(Sn * me);
    eta_t = ceta * sqrt(St * me);
  } else {
    linear_constants_d(Re, me, Ye, lin[0], lin[1], &kn, &eta_n);
    kt = kn;
    eta_t = eta_n;
  }
  double Fn[3], Ft[3];
  for (int d = 0; d < 3; d++) {
    Fn[d] = -(kn * dn) * nrm[d] - eta_n * vrn[d];
    Ft[d] = -(kt * H[d]) - eta_t * vrt[d];
  }
  double aFn = sqrt(dot3d(Fn, Fn));
  double aFt = sqrt(dot3d(Ft, Ft));
  if (aFt > 0.0 && aFt >= mu * aFn) {
    for (int d = 0; d < 3; d++) {
      Ft[d] = mu * aFn * Ft[d] / aFt;
      H[d] = (Ft[d] + eta_t * vrt[d]) / (-kt);
    }
  }
  cross3d(nrm, Ft, nxFt);
  Mr[0] = Mr[1] = Mr[2] = 0.0;
  double adw = sqrt(dot3d(dw, dw));
  if (rolling == 1 && adw > 0.0)
    for (int d = 0; d < 3; d++) Mr[d] = -mur * Re * aFn * dw[d] / adw;
  if (rolling == 2 && adw > 0.0) {
    const double avw = sqrt(dot3d(vom, vom));
    for (int d = 0; d < 3; d++) Mr[d] = -mur * Re * aFn * avw * dw[d] / adw;
  }
  for (int d = 0; d < 3; d++) Fsum[d] = Fn[d] + Ft[d];
}

// A translating wall where its motion has carried it by time t.
__device__ __forceinline__ WallDev wall_at(const WallDev& W, double t) {
  WallDev o = W;
  if (W.translates)
    for (int d = 0; d < 3; d++) {
      o.p[d] = W.p[d] + W.V[d] * t;
      o.c[d] = W.c[d] + W.V[d] * t;
    }
  return o;
}

// Nearest wall point and normal overlap in FP64 (same statements as the CPU reference).
__device__ __forceinline__ bool wall_geom_d(const WallDev& W, const double* x, double R, double* nrm,
                                            double* dn, double* ps) {
  if (W.kind == 0) {
    double rel[3] = {x[0] - W.p[0], x[1] - W.p[1], x[2] - W.p[2]};
    double dist = dot3d(rel, W.n);
    double ov = R - dist;
    if (!(ov > 0.0)) return false;
    for (int d = 0; d < 3; d++) {
      nrm[d] = -W.n[d];
      ps[d] = x[d] - dist * W.n[d];
    }
    *dn = ov;
    return true;
  }
  if (W.kind == 1) {
    double rel[3] = {x[0] - W.p[0], x[1] - W.p[1], x[2] - W.p[2]};
    double ax = dot3d(rel, W.n);
    double rad[3] = {rel[0] - ax * W.n[0], rel[1] - ax * W.n[1], rel[2] - ax * W.n[2]};
    double rho = sqrt(dot3d(rad, rad));
    if (!(rho > 0.0)) return false;
    double ov = R - (W.radius - rho);
    if (!(ov > 0.0)) return false;
    for (int d = 0; d < 3; d++) {
      nrm[d] = rad[d] / rho;
      ps[d] = W.p[d] + ax * W.n[d] + W.radius * nrm[d];
    }
    *dn = ov;
    return true;
  }
  if (W.kind == 2) {
    double rel[3] = {x[0] - W.p[0], x[1] - W.p[1], x[2] - W.p[2]};
    double h = dot3d(rel, W.n);
    double q[3] = {rel[0] - h * W.n[0], rel[1] - h * W.n[1], rel[2] - h * W.n[2]};
    double rho = sqrt(dot3d(q, q));
    double loc[3];
    if (rho < W.inner || rho > W.radius) {
      double target = rho < W.inner ? W.inner : W.radius;
      double u[3];
      if (rho > 0.0) {
        for (int d = 0; d < 3; d++) u[d] = q[d] / rho;
      } else {
        double e[3] = {1.0, 0.0, 0.0};
        if (fabs(W.n[0]) > 0.9) {
          e[0] = 0.0;
          e[1] = 1.0;
        }
        double c = dot3d(e, W.n);
        for (int d = 0; d < 3; d++) u[d] = e[d] - c * W.n[d];
        double nu = sqrt(dot3d(u, u));
        for (int d = 0; d < 3; d++) u[d] /= nu;
      }
      for (int d = 0; d < 3; d++) loc[d] = target * u[d];
    } else {
      for (int d = 0; d < 3; d++) loc[d] = q[d];
    }
    double D[3];
    for (int d = 0; d < 3; d++) {
      ps[d] = W.p[d] + loc[d];
      D[d] = ps[d] - x[d];
    }
    double dist = sqrt(dot3d(D, D));
    double ov = R - dist;
    if (!(ov > 0.0) || !(dist > 0.0)) return false;
    for (int d = 0; d < 3; d++) nrm[d] = D[d] / dist;
    *dn = ov;
    return true;
  }
  return false;
}

// Conservative FP32 test that a wall may touch a sphere at (approximately) xf.
__device__ __forceinline__ bool wall_maybe_f(int kind, const WallF& W, const float* xf, float R, float margin) {
  float rel[3] = {xf[0] - W.p[0], xf[1] - W.p[1], xf[2] - W.p[2]};
  float h = rel[0] * W.n[0] + rel[1] * W.n[1] + rel[2] * W.n[2];
  if (kind == 0) return h < R + margin;
  float q[3] = {rel[0] - h * W.n[0], rel[1] - h * W.n[1], rel[2] - h * W.n[2]};
  float rho = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
  if (kind == 1) return W.radius - rho < R + margin;
  // annulus: distance to the ring = sqrt(h^2 + radial gap outside the ring^2)
  float gap = fmaxf(fmaxf(W.inner - rho, rho - W.radius), 0.0f);
  return h * h + gap * gap < (R + margin) * (R + margin);
}

// ------------------------------------------------------------------ FP32 contact law
// kExt: the paper's other options (linear model, viscous rolling) may occur; without it
// they are compiled out, and the kernel keeps the registers of the default model.
// Outputs the pieces of one contact: Fp = F_n + F_t on the particle, n x F_t (times the
// lever R_i on the particle, R_j on its partner) and the rolling torque M_r (on the
// partner: -M_r, Table rolling_torque's w_ji = -w_ij).
template <bool kExt>
__device__ __forceinline__ void law_pieces_f(const float* nrm, float dn, const float* vij, const float* dw,
                                             const float* vom, float Re, float me, float Ye, float Ge, float ceta,
                                             float mu, float mur, int rolling, const float* lin, float dt, double* H,
                                             bool incr, float* Fp, float* nxFt, float* Mr) {
  float vn = vij[0] * nrm[0] + vij[1] * nrm[1] + vij[2] * nrm[2];
  float vrn[3], vrt[3];
  for (int d = 0; d < 3; d++) {
    vrn[d] = vn * nrm[d];
    vrt[d] = vij[d] - vrn[d];
  }
  // tangential overlap accumulated in FP64 (Eq. delta_t)
  if (incr)
    for (int d = 0; d < 3; d++) H[d] = H[d] + f2d_int(vrt[d] * dt);
  float Hf[3] = {d2f_int(H[0]), d2f_int(H[1]), d2f_int(H[2])};
  float kn, kt, eta_n, eta_t;
  if (!kExt || lin == nullptr) {
    const float sq = sqrtf(Re * dn);
    kn = (4.0f / 3.0f) * Ye * sq;
    const float Sn = 2.0f * Ye * sq;
    kt = 8.0f * Ge * sq;
    eta_n = ceta * sqrtf(Sn * me);
    eta_t = ceta * sqrtf(kt * me);
  } else {  // Eqs. linearkn, linearetan
    const float sR = sqrtf(Re);
    kn = (16.0f / 15.0f) * sR * Ye * powf(15.0f * me * lin[0] * lin[0] / (16.0f * sR * Ye), 0.2f);
    eta_n = sqrtf(4.0f * me * kn / lin[1]);
    kt = kn;
    eta_t = eta_n;
  }
  float Fn[3], Ft[3];
  for (int d = 0; d < 3; d++) {
    Fn[d] = -(kn * dn) * nrm[d] - eta_n * vrn[d];
    Ft[d] = -(kt * Hf[d]) - eta_t * vrt[d];
  }
  float aFn = sqrtf(Fn[0] * Fn[0] + Fn[1] * Fn[1] + Fn[2] * Fn[2]);
  float aFt = sqrtf(Ft[0] * Ft[0] + Ft[1] * Ft[1] + Ft[2] * Ft[2]);
  if (aFt > 0.0f && aFt >= mu * aFn) {
    float s = mu * aFn / aFt;
    float ikt = -1.0f / kt;
    for (int d = 0; d < 3; d++) {
      Ft[d] = s * Ft[d];
      H[d] = f2d_int((Ft[d] + eta_t * vrt[d]) * ikt);
    }
  }
  nxFt[0] = nrm[1] * Ft[2] - nrm[2] * Ft[1];
  nxFt[1] = nrm[2] * Ft[0] - nrm[0] * Ft[2];
  nxFt[2] = nrm[0] * Ft[1] - nrm[1] * Ft[0];
  Mr[0] = Mr[1] = Mr[2] = 0.f;
  if (rolling == 1 && (dw[0] != 0.f || dw[1] != 0.f || dw[2] != 0.f)) {
    // unit vector of w_i - w_j, scaled first so that tiny relative spins do not underflow
    const float s = 1.0f / fmaxf(fmaxf(fabsf(dw[0]), fabsf(dw[1])), fabsf(dw[2]));
    const float u[3] = {dw[0] * s, dw[1] * s, dw[2] * s};
    float c = -mur * Re * aFn * rsqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int d = 0; d < 3; d++) Mr[d] = c * u[d];
  }
  if (kExt && rolling == 2 && (dw[0] != 0.f || dw[1] != 0.f || dw[2] != 0.f)) {
    const float s = 1.0f / fmaxf(fmaxf(fabsf(dw[0]), fabsf(dw[1])), fabsf(dw[2]));
    const float u[3] = {dw[0] * s, dw[1] * s, dw[2] * s};
    const float avw = sqrtf(vom[0] * vom[0] + vom[1] * vom[1] + vom[2] * vom[2]);
    const float c = -mur * Re * aFn * avw * rsqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int d = 0; d < 3; d++) Mr[d] = c * u[d];
  }
  for (int d = 0; d < 3; d++) Fp[d] = Fn[d] + Ft[d];
}

// One contact added to the particle's sums: F += F_n + F_t, M += R_i n x F_t + M_r.
template <bool kExt>
__device__ __forceinline__ void law_f(const float* nrm, float dn, const float* vij, const float* dw,
                                      const float* vom, float Re, float me, float Ye, float Ge, float ceta,
                                      float mu, float mur, int rolling, const float* lin, float dt, double* H,
                                      bool incr, float Ri, float* F, float* M) {
  float Fp[3], nxFt[3], Mr[3];
  law_pieces_f<kExt>(nrm, dn, vij, dw, vom, Re, me, Ye, Ge, ceta, mu, mur, rolling, lin, dt, H, incr, Fp, nxFt, Mr);
  for (int d = 0; d < 3; d++) {
    F[d] += Fp[d];
    M[d] += Ri * nxFt[d] + Mr[d];
  }
}

// ------------------------------------------------------------------ block statistics
struct StepStats {
  unsigned touch, wtouch, active;
  float max_ovl;
  unsigned status;
};

__device__ __forceinline__ void block_flush(const StepStats& s, Control* C) {
  __shared__ unsigned sh_t, sh_w, sh_a, sh_st;
  __shared__ float sh_o;
  if (threadIdx.x == 0) {
    sh_t = 0; sh_w = 0; sh_a = 0; sh_st = 0; sh_o = 0.0f;
  }
  __syncthreads();
  unsigned t = s.touch, w = s.wtouch, a = s.active, st = s.status;
  float o = s.max_ovl;
  for (int off = 16; off > 0; off >>= 1) {
    t += __shfl_down_sync(0xffffffffu, t, off);
    w += __shfl_down_sync(0xffffffffu, w, off);
    a += __shfl_down_sync(0xffffffffu, a, off);
    st |= __shfl_down_sync(0xffffffffu, st, off);
    o = fmaxf(o, __shfl_down_sync(0xffffffffu, o, off));
  }
  if ((threadIdx.x & 31) == 0) {
    if (t) atomicAdd(&sh_t, t);
    if (w) atomicAdd(&sh_w, w);
    if (a) atomicAdd(&sh_a, a);
    if (st) atomicOr(&sh_st, st);
    atomicMax((unsigned*)&sh_o, __float_as_uint(o));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (sh_t) atomicAdd(&C->n_touch_dir, (unsigned long long)sh_t);
    if (sh_w) atomicAdd(&C->n_wall_touch, (unsigned long long)sh_w);
    if (sh_a) atomicAdd(&C->n_active, (unsigned long long)sh_a);
    if (sh_st) atomicOr(&C->status, sh_st);
    atomicMax(&C->max_ovl_bits, __float_as_uint(sh_o));
  }
}

// End of an evaluation.  The counters of dem_get_stats describe the last evaluation of a
// dem_step call, so only that one reduces them; the others publish error bits alone (rare,
// one atomic per failing thread).  The parities of the state and the history flip after
// the kernel: it only marks the flip as due (a plain store of one thread), and the next
// k_begin or the k_end closing the call applies it (apply_flip), so no block waits on a
// grid-wide count.  A step made of two kernels marks it from the second only.
__device__ __forceinline__ void end_step(const StepStats& st, Control* C, bool last, bool closes_step = true) {
  if (last)
    block_flush(st, C);
  else if (st.status)
    atomicOr(&C->status, st.status);
  if (closes_step && blockIdx.x == 0 && threadIdx.x == 0) C->flip_due = 1;
}

// Exact "z < z_sink" on FP64 values with integer operations.
__device__ __forceinline__ bool below_sink(double z, long long sink_key) {
  return ordered_key(__double_as_longlong(z)) < sink_key;
}

__device__ __forceinline__ bool finite_d(double x) {
  return ((unsigned)__double2hiint(x) & 0x7FF00000u) != 0x7FF00000u;
}

}  // namespace demgb
