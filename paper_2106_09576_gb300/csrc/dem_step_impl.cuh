// dem_step_impl.cuh -- the per-time-step kernel: particle-particle and particle-wall
// contact forces, tangential-overlap history, and velocity Verlet (Sec. 2.1-2.2).
//
// One thread owns one particle i of the cell-sorted order.  It walks i's fine-search
// list (ordered by partner id, so the force sums run in the same order as a serial
// loop over pairs in id order), evaluates every touching contact from i's side, sums
// F_i and M_i in registers (no atomics; each pair is evaluated by both partners, which
// give bitwise opposite results), then integrates:
//   v^{n}   = v^{n-1/2} + a^n dt/2     (Eq. newvv)
//   v^{n+1/2} = v^n + a^n dt/2          (Eq. halfstep, next step)
//   x^{n+1} = x^n + v^{n+1/2} dt
// and flags a contact search when |x^{n+1} - x_ref| > skin/2 (dynamic mode, Sec. 3.1).
//
// MIXED = false: every operation in FP64, in the order of the CPU reference; this
//   translation unit is compiled without FMA contraction.
// MIXED = true: relative positions are formed exactly as FP32 pairs from integer splits
//   of the FP64 positions; the normal overlap uses a double-float difference of squares
//   (S^2 - r^2) / (S + r); the contact law runs in FP32; the tangential overlap is
//   accumulated and stored in FP64; integration is FP64.  FP64 instructions per
//   particle-step: 9 for integration plus 3 per touching contact.
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

__device__ __forceinline__ void law_d(const double* nrm, double dn, const double* vij, const double* dw,
                                      double Re, double me, double Ye, double Ge, double ceta, double mu,
                                      double mur, int rolling, double dt, double* H, bool incr, double* Fsum,
                                      double* nxFt, double* Mr) {
  double vn = dot3d(vij, nrm);
  double vrn[3], vrt[3];
  for (int d = 0; d < 3; d++) {
    vrn[d] = vn * nrm[d];
    vrt[d] = vij[d] - vrn[d];
  }
  if (incr)
    for (int d = 0; d < 3; d++) H[d] = H[d] + vrt[d] * dt;
  double sq = sqrt(Re * dn);
  double kn = 4.0 / 3.0 * Ye * sq;
  double Sn = 2.0 * Ye * sq;
  double kt = 8.0 * Ge * sq;
  double St = 8.0 * Ge * sq;
  double eta_n = ceta * sqrt(Sn * me);
  double eta_t = ceta * sqrt(St * me);
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
  for (int d = 0; d < 3; d++) Fsum[d] = Fn[d] + Ft[d];
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

// Conservative FP32 test that wall W may touch a sphere at (approximately) xf.
__device__ __forceinline__ bool wall_maybe_f(const WallDev& W, const float* xf, float R, float margin) {
  float rel[3] = {xf[0] - (float)W.p[0], xf[1] - (float)W.p[1], xf[2] - (float)W.p[2]};
  float h = rel[0] * (float)W.n[0] + rel[1] * (float)W.n[1] + rel[2] * (float)W.n[2];
  if (W.kind == 0) return h < R + margin;
  float q[3] = {rel[0] - h * (float)W.n[0], rel[1] - h * (float)W.n[1], rel[2] - h * (float)W.n[2]};
  float rho = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
  if (W.kind == 1) return (float)W.radius - rho < R + margin;
  // annulus: distance to the ring >= max(|h|, radial gap outside the ring)
  float gap = fmaxf(fmaxf((float)W.inner - rho, rho - (float)W.radius), 0.0f);
  return h * h + gap * gap < (R + margin) * (R + margin);
}

// ------------------------------------------------------------------ FP32 contact law
__device__ __forceinline__ void law_f(const float* nrm, float dn, const float* vij, const float* dw, float Re,
                                      float me, float Ye, float Ge, float ceta, float mu, float mur,
                                      int rolling, float dt, double* H, bool incr, float Ri, float* F,
                                      float* M) {
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
  float sq = sqrtf(Re * dn);
  float kn = (4.0f / 3.0f) * Ye * sq;
  float Sn = 2.0f * Ye * sq;
  float kt = 8.0f * Ge * sq;
  float eta_n = ceta * sqrtf(Sn * me);
  float eta_t = ceta * sqrtf(kt * me);
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
  float nxFt[3] = {nrm[1] * Ft[2] - nrm[2] * Ft[1], nrm[2] * Ft[0] - nrm[0] * Ft[2],
                   nrm[0] * Ft[1] - nrm[1] * Ft[0]};
  float Mr[3] = {0.f, 0.f, 0.f};
  float adw2 = dw[0] * dw[0] + dw[1] * dw[1] + dw[2] * dw[2];
  if (rolling == 1 && adw2 > 0.0f) {
    float c = -mur * Re * aFn * rsqrtf(adw2);
    for (int d = 0; d < 3; d++) Mr[d] = c * dw[d];
  }
  for (int d = 0; d < 3; d++) {
    F[d] += Fn[d] + Ft[d];
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

// ------------------------------------------------------------------ the step kernel
template <bool MIXED>
__global__ void __launch_bounds__(kStepBlock) k_step(Params P) {
  const Control* C = P.ctl;
  const int cur = C->cur, nxt = cur ^ 1, sb = C->sbuf, hc = C->hc;
  const bool init = C->init != 0, last = C->last != 0;
  const int n = P.n, nact = C->n_act_sorted;
  const double t_now = (double)C->step * P.dt;   // time of this force evaluation
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  StepStats st = {0u, 0u, 0u, 0.0f, 0u};

  if (i < nact) {
    const double* X = P.x[cur];
    const double* V = P.v[cur];
    const double* W = P.w[cur];
    const uint8_t* A = P.act[cur];
    const float* RAD = P.rad[sb];
    double* Xo = P.x[nxt];
    double* Vo = P.v[nxt];
    double* Wo = P.w[nxt];
    double xi[3] = {X[i], X[n + i], X[2 * n + i]};
    double vi[3] = {V[i], V[n + i], V[2 * n + i]};
    double wi[3] = {W[i], W[n + i], W[2 * n + i]};
    unsigned long long mnew = 0ull;
    if (!A[i]) {
      // left the system since the last rebuild: frozen
      for (int d = 0; d < 3; d++) {
        Xo[d * n + i] = xi[d];
        Vo[d * n + i] = vi[d];
        Wo[d * n + i] = wi[d];
        if (last) {
          P.out_v[d * n + i] = vi[d];
          P.out_w[d * n + i] = wi[d];
          P.out_F[d * n + i] = 0.0;
          P.out_M[d * n + i] = 0.0;
        }
      }
      P.act[nxt][i] = 0;
      P.mask[hc ^ 1][i] = 0ull;
    } else {
      const unsigned long long mold = P.mask[hc][i];
      const double* Hold = P.hist[hc] + (size_t)i * kHistStride * 3;
      double* Hnew = P.hist[hc ^ 1] + (size_t)i * kHistStride * 3;
      const int* nb = P.nbr + (size_t)i * kMaxNbr;
      const int cnt = P.nbr_cnt[i];
      int rank = 0;
      const float Rif = RAD[i];
      const double Ri = (double)Rif;
      double Fd[3] = {0.0, 0.0, 0.0}, Md[3] = {0.0, 0.0, 0.0};
      float Ff[3] = {0.f, 0.f, 0.f}, Mf[3] = {0.f, 0.f, 0.f};
      float hx[3], lx[3], vif[3], wif[3];
      double mi_d = 0.0, Ii_d = 0.0;
      float mi_f = 0.f;
      if (MIXED) {
        for (int d = 0; d < 3; d++) {
          split_df(xi[d], hx[d], lx[d]);
          vif[d] = d2f_int(vi[d]);
          wif[d] = d2f_int(wi[d]);
        }
        mi_f = (float)P.density * (4.0f / 3.0f) * 3.14159265358979f * Rif * Rif * Rif;
      } else {
        mi_d = P.density * (4.0 / 3.0) * 3.14159265358979323846 * Ri * Ri * Ri;
        Ii_d = 0.4 * mi_d * Ri * Ri;
      }

      // ---------------- particle-particle contacts, list order (partner id order)
      for (int k = 0; k < cnt; k++) {
        const int j = nb[k];
        const bool had = (mold >> k) & 1ull;
        if (!A[j]) continue;
        const float Rjf = RAD[j];
        if (MIXED) {
          float s[3], t[3], dxf[3];
          float hj, lj;
          for (int d = 0; d < 3; d++) {
            split_df(X[d * n + j], hj, lj);
            df_diff(hx[d], lx[d], hj, lj, s[d], t[d]);
            dxf[d] = s[d] + t[d];
          }
          const float S = Rif + Rjf;
          const float r2f = dxf[0] * dxf[0] + dxf[1] * dxf[1] + dxf[2] * dxf[2];
          if (!(r2f < S * S * 1.000001f)) continue;
          // exact S^2 - r^2 as a double-float
          float p, pe, Ah, Al, e;
          two_prod(s[0], s[0], Ah, pe);
          Al = pe + (2.0f * s[0] + t[0]) * t[0];
          two_prod(s[1], s[1], p, pe);
          two_sum(Ah, p, Ah, e);
          Al += e + pe + (2.0f * s[1] + t[1]) * t[1];
          two_prod(s[2], s[2], p, pe);
          two_sum(Ah, p, Ah, e);
          Al += e + pe + (2.0f * s[2] + t[2]) * t[2];
          float Sh, Sl, P2, P2e, Dh, De;
          two_sum(Rif, Rjf, Sh, Sl);
          two_prod(Sh, Sh, P2, P2e);
          P2e += 2.0f * Sh * Sl;
          two_sum(P2, -Ah, Dh, De);
          const float D = Dh + (De + (P2e - Al));
          if (!(D > 0.0f)) continue;
          const float r = sqrtf(Ah + Al);
          const float dn = D / (Sh + r);
          const float ir = 1.0f / r;
          const float nrm[3] = {dxf[0] * ir, dxf[1] * ir, dxf[2] * ir};
          float vjf[3], wjf[3];
          for (int d = 0; d < 3; d++) {
            vjf[d] = d2f_int(V[d * n + j]);
            wjf[d] = d2f_int(W[d * n + j]);
          }
          const float rw[3] = {Rif * wif[0] + Rjf * wjf[0], Rif * wif[1] + Rjf * wjf[1],
                               Rif * wif[2] + Rjf * wjf[2]};
          const float vij[3] = {(vif[0] - vjf[0]) + (rw[1] * nrm[2] - rw[2] * nrm[1]),
                                (vif[1] - vjf[1]) + (rw[2] * nrm[0] - rw[0] * nrm[2]),
                                (vif[2] - vjf[2]) + (rw[0] * nrm[1] - rw[1] * nrm[0])};
          const float dw[3] = {wif[0] - wjf[0], wif[1] - wjf[1], wif[2] - wjf[2]};
          const float Re = Rif * Rjf / S;
          const float mj = (float)P.density * (4.0f / 3.0f) * 3.14159265358979f * Rjf * Rjf * Rjf;
          const float me = mi_f * mj / (mi_f + mj);
          double H[3] = {0.0, 0.0, 0.0};
          if (had) {
            const int ro = __popcll(mold & ((1ull << k) - 1ull));
            H[0] = Hold[ro * 3];
            H[1] = Hold[ro * 3 + 1];
            H[2] = Hold[ro * 3 + 2];
          }
          law_f(nrm, dn, vij, dw, Re, me, (float)P.Ye_pp, (float)P.Ge_pp, (float)P.ceta_pp, (float)P.mu_pp,
                (float)P.mur_pp, P.rolling, (float)P.dt, H, !init, Rif, Ff, Mf);
          st.touch++;
          st.max_ovl = fmaxf(st.max_ovl, dn / fminf(Rif, Rjf));
          if (rank < kHistStride) {
            Hnew[rank * 3] = H[0];
            Hnew[rank * 3 + 1] = H[1];
            Hnew[rank * 3 + 2] = H[2];
            mnew |= 1ull << k;
            rank++;
          } else {
            st.status |= kStCapacity;
          }
        } else {
          const double xj[3] = {X[j], X[n + j], X[2 * n + j]};
          const double Rj = (double)Rjf;
          const double r = sqrt(sqdist_exact(xi[0], xi[1], xi[2], xj[0], xj[1], xj[2]));
          const double dn = (Ri + Rj) - r;
          if (!(dn > 0.0)) continue;
          const double dx[3] = {xj[0] - xi[0], xj[1] - xi[1], xj[2] - xi[2]};
          const double nrm[3] = {dx[0] / r, dx[1] / r, dx[2] / r};
          const double vj[3] = {V[j], V[n + j], V[2 * n + j]};
          const double wj[3] = {W[j], W[n + j], W[2 * n + j]};
          double rw[3], rwxn[3], vij[3], dw[3];
          for (int d = 0; d < 3; d++) rw[d] = Ri * wi[d] + Rj * wj[d];
          cross3d(rw, nrm, rwxn);
          for (int d = 0; d < 3; d++) {
            vij[d] = (vi[d] - vj[d]) + rwxn[d];
            dw[d] = wi[d] - wj[d];
          }
          const double Re = 1.0 / (1.0 / Ri + 1.0 / Rj);
          const double mj = P.density * (4.0 / 3.0) * 3.14159265358979323846 * Rj * Rj * Rj;
          const double me = 1.0 / (1.0 / mi_d + 1.0 / mj);
          double H[3] = {0.0, 0.0, 0.0};
          if (had) {
            const int ro = __popcll(mold & ((1ull << k) - 1ull));
            H[0] = Hold[ro * 3];
            H[1] = Hold[ro * 3 + 1];
            H[2] = Hold[ro * 3 + 2];
          }
          double f[3], nxFt[3], Mr[3];
          law_d(nrm, dn, vij, dw, Re, me, P.Ye_pp, P.Ge_pp, P.ceta_pp, P.mu_pp, P.mur_pp, P.rolling, P.dt, H,
                !init, f, nxFt, Mr);
          for (int d = 0; d < 3; d++) {
            Fd[d] += f[d];
            Md[d] += Ri * nxFt[d] + Mr[d];
          }
          st.touch++;
          st.max_ovl = fmaxf(st.max_ovl, (float)(dn / fmin(Ri, Rj)));
          if (rank < kHistStride) {
            Hnew[rank * 3] = H[0];
            Hnew[rank * 3 + 1] = H[1];
            Hnew[rank * 3 + 2] = H[2];
            mnew |= 1ull << k;
            rank++;
          } else {
            st.status |= kStCapacity;
          }
        }
      }

      // ---------------- particle-wall contacts (Sec. 2.1 last paragraph; Sec. 3.6)
      for (int k = 0; k < P.n_walls; k++) {
        const WallDev& Wl = P.walls[k];
        if (!(t_now >= Wl.t_on && t_now < Wl.t_off)) continue;
        if (MIXED) {
          const float xf[3] = {hx[0] + lx[0], hx[1] + lx[1], hx[2] + lx[2]};
          if (!wall_maybe_f(Wl, xf, Rif, P.wall_margin)) continue;
        }
        double nrm[3], dn, ps[3];
        if (!wall_geom_d(Wl, xi, Ri, nrm, &dn, ps)) continue;
        double arm[3] = {ps[0] - Wl.c[0], ps[1] - Wl.c[1], ps[2] - Wl.c[2]};
        double Vw[3];
        cross3d(Wl.Om, arm, Vw);
        for (int d = 0; d < 3; d++) Vw[d] += Wl.V[d];
        const int bit = 56 + k;
        double H[3] = {0.0, 0.0, 0.0};
        if ((mold >> bit) & 1ull) {
          const int ro = __popcll(mold & ((1ull << bit) - 1ull));
          H[0] = Hold[ro * 3];
          H[1] = Hold[ro * 3 + 1];
          H[2] = Hold[ro * 3 + 2];
        }
        if (MIXED) {
          const float nf[3] = {(float)nrm[0], (float)nrm[1], (float)nrm[2]};
          const float dnf = (float)dn;
          const float Vwf[3] = {(float)Vw[0], (float)Vw[1], (float)Vw[2]};
          const float rw[3] = {Rif * wif[0], Rif * wif[1], Rif * wif[2]};
          const float vij[3] = {(vif[0] - Vwf[0]) + (rw[1] * nf[2] - rw[2] * nf[1]),
                                (vif[1] - Vwf[1]) + (rw[2] * nf[0] - rw[0] * nf[2]),
                                (vif[2] - Vwf[2]) + (rw[0] * nf[1] - rw[1] * nf[0])};
          const float dw[3] = {wif[0] - (float)Wl.Om[0], wif[1] - (float)Wl.Om[1], wif[2] - (float)Wl.Om[2]};
          law_f(nf, dnf, vij, dw, Rif, mi_f, (float)P.Ye_pw, (float)P.Ge_pw, (float)P.ceta_pw, (float)P.mu_pw,
                (float)P.mur_pw, P.rolling, (float)P.dt, H, !init, Rif, Ff, Mf);
          st.max_ovl = fmaxf(st.max_ovl, dnf / Rif);
        } else {
          double rw[3], rwxn[3], vij[3], dw[3];
          for (int d = 0; d < 3; d++) rw[d] = Ri * wi[d];
          cross3d(rw, nrm, rwxn);
          for (int d = 0; d < 3; d++) {
            vij[d] = (vi[d] - Vw[d]) + rwxn[d];
            dw[d] = wi[d] - Wl.Om[d];
          }
          double f[3], nxFt[3], Mr[3];
          law_d(nrm, dn, vij, dw, Ri, mi_d, P.Ye_pw, P.Ge_pw, P.ceta_pw, P.mu_pw, P.mur_pw, P.rolling, P.dt, H,
                !init, f, nxFt, Mr);
          for (int d = 0; d < 3; d++) {
            Fd[d] += f[d];
            Md[d] += Ri * nxFt[d] + Mr[d];
          }
          st.max_ovl = fmaxf(st.max_ovl, (float)(dn / Ri));
        }
        st.wtouch++;
        if (rank < kHistStride) {
          Hnew[rank * 3] = H[0];
          Hnew[rank * 3 + 1] = H[1];
          Hnew[rank * 3 + 2] = H[2];
          mnew |= 1ull << bit;
          rank++;
        } else {
          st.status |= kStCapacity;
        }
      }
      P.mask[hc ^ 1][i] = mnew;

      // ---------------- integration (Eqs. main1, main2, halfstep, newvv)
      double xn[3], vn[3], wn[3];
      if (MIXED) {
        const float mi = mi_f;
        const float inv_m = 1.0f / mi;
        const float inv_I = 1.0f / (0.4f * mi * Rif * Rif);
        for (int d = 0; d < 3; d++) {
          const double a = f2d_int(Ff[d] * inv_m + (float)P.g[d]);
          const double al = f2d_int(Mf[d] * inv_I);
          if (init) {
            vn[d] = fma(a, P.half_dt, vi[d]);
            wn[d] = fma(al, P.half_dt, wi[d]);
          } else {
            vn[d] = fma(a, P.dt, vi[d]);
            wn[d] = fma(al, P.dt, wi[d]);
          }
          if (last) {
            P.out_v[d * n + i] = init ? vi[d] : fma(a, P.half_dt, vi[d]);
            P.out_w[d * n + i] = init ? wi[d] : fma(al, P.half_dt, wi[d]);
            P.out_F[d * n + i] = (double)Ff[d];
            P.out_M[d * n + i] = (double)Mf[d];
          }
          xn[d] = fma(vn[d], P.dt, xi[d]);
        }
      } else {
        const double h = P.half_dt;
        for (int d = 0; d < 3; d++) {
          const double a = Fd[d] / mi_d + P.g[d];
          const double al = Md[d] / Ii_d;
          double vf = vi[d], wf = wi[d];
          if (!init) {
            vf = vf + a * h;
            wf = wf + al * h;
          }
          if (last) {
            P.out_v[d * n + i] = vf;
            P.out_w[d * n + i] = wf;
            P.out_F[d * n + i] = Fd[d];
            P.out_M[d * n + i] = Md[d];
          }
          vn[d] = vf + a * h;
          wn[d] = wf + al * h;
          xn[d] = xi[d] + vn[d] * P.dt;
        }
      }
      bool alive = !(xn[2] < P.z_sink);
      for (int d = 0; d < 3; d++) {
        Xo[d * n + i] = xn[d];
        Vo[d * n + i] = vn[d];
        Wo[d * n + i] = wn[d];
      }
      P.act[nxt][i] = alive ? 1 : 0;
      if (!(isfinite(xn[0]) && isfinite(xn[1]) && isfinite(xn[2]) && isfinite(vn[0]) && isfinite(vn[1]) &&
            isfinite(vn[2])))
        st.status |= kStNonfinite;
      if (alive) {
        st.active++;
        // dynamic contact-search trigger: |x^{n+1} - x_ref|^2 > (skin/2)^2 (Sec. 3.1)
        const double xr[3] = {P.xref[i], P.xref[n + i], P.xref[2 * n + i]};
        bool far;
        if (MIXED) {
          float d2 = 0.f;
          for (int d = 0; d < 3; d++) {
            float ah, al, bh, bl, s, t;
            split_df(xr[d], ah, al);
            split_df(xn[d], bh, bl);
            df_diff(ah, al, bh, bl, s, t);
            const float u = s + t;
            d2 += u * u;
          }
          far = d2 > (float)P.disp_lim2 * 0.99999f;
        } else {
          far = sqdist_exact(xr[0], xr[1], xr[2], xn[0], xn[1], xn[2]) > P.disp_lim2;
        }
        if (far && P.rebuild_every <= 0) P.ctl->need_rebuild = 1;
      }
    }
  }
  if (P.max_overlap_ratio > 0.0 && st.max_ovl > (float)P.max_overlap_ratio) st.status |= kStOverlap;
  block_flush(st, P.ctl);
  // The last block to finish flips the state and history parities: every block has
  // read them by then.
  __shared__ bool is_last;
  __threadfence();
  if (threadIdx.x == 0) is_last = atomicAdd(&P.ctl->blocks_done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    Control* Cw = P.ctl;
    Cw->cur ^= 1;
    Cw->hc ^= 1;
    Cw->init = 0;
    Cw->ran = 1;
    Cw->blocks_done = 0;
    __threadfence();
  }
}

}  // namespace demgb
