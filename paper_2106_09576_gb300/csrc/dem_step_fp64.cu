// dem_step_fp64.cu -- the FP64 step kernel (forces, history, integration), built with
// -fmad=false so that every product and sum rounds separately.
//
// One thread owns one particle i of the cell-sorted order.  It walks i's fine-search list
// (ordered by partner id), evaluates each touching contact from i's side with the same
// operations as the serial statement of Sec. 2.1 and adds it to F_i, M_i in list order,
// then the walls in wall order: the sums therefore run in the same order as a serial loop
// over pairs (i < j) in id order, and each pair term from j's side is the exact negation
// of the term from i's side.  The results are bit-identical to that serial loop.
#include "dem_step_common.cuh"

namespace demgb {

template <bool kBatch>
__global__ void __launch_bounds__(kStepBlock) k_step_fp64(const __grid_constant__ Params P) {
  const Control* C = P.ctl;
  const int cur = C->cur, nxt = cur ^ 1, sb = C->sbuf, hc = C->hc;
  const bool init = C->init != 0, last = C->last != 0;
  const unsigned wall_on = C->wall_on;
  const int n = P.n, nact = C->n_act_sorted;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  StepStats st = {0u, 0u, 0u, 0.0f, 0u};

  if (last && i >= nact && i < n) {
    for (int d = 0; d < 3; d++) {   // out of the system: frozen in both buffers
      P.out_v[d * n + i] = P.v[cur][d * n + i];
      P.out_w[d * n + i] = P.w[cur][d * n + i];
      P.out_F[d * n + i] = 0.0;
      P.out_M[d * n + i] = 0.0;
    }
  }
  if (i < nact) {
    const double* X = P.x[cur];
    const double* V = P.v[cur];
    const double* W = P.w[cur];
    const uint8_t* A = P.act[cur];
    const float* RAD = P.rad[sb];
    double* Xo = P.x[nxt];
    double* Vo = P.v[nxt];
    double* Wo = P.w[nxt];
    const double xi[3] = {X[i], X[n + i], X[2 * n + i]};
    const double vi[3] = {V[i], V[n + i], V[2 * n + i]};
    const double wi[3] = {W[i], W[n + i], W[2 * n + i]};
    if (!A[i]) {
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
      const double* Hold = P.hist[hc] + (size_t)i;
      double* Hnew = P.hist[hc ^ 1] + (size_t)i;
      const int* nb = P.nbr + (size_t)i * kMaxNbr;
      const int cnt = P.nbr_cnt[i];
      unsigned long long mnew = 0ull;
      int rank = 0;
      // materials and walls: the context's, or those of the particle's instance in a batch
      const InstDev* I = kBatch ? P.itab + P.inst[sb][i] : nullptr;
      const MatD& Mt = kBatch ? I->md : P.md;
      const WallDev* WLs = kBatch ? I->walls : P.walls;
      const int n_walls = kBatch ? I->n_walls : P.n_walls;
      unsigned won = wall_on;
      if (kBatch) {
        won = 0u;
        const double t = (double)C->step * P.dt;
        for (int k = 0; k < n_walls; k++)
          if (t >= WLs[k].t_on && t < WLs[k].t_off) won |= 1u << k;
      }
      const bool lin = P.contact_model == 1;
      const double lin_pp[2] = {P.lin_V, Mt.lin_den_pp}, lin_pw[2] = {P.lin_V, Mt.lin_den_pw};
      const double Ri = (double)RAD[i];
      const double mi = P.density * (4.0 / 3.0) * 3.14159265358979323846 * Ri * Ri * Ri;
      const double Ii = 0.4 * mi * Ri * Ri;
      double F[3] = {0.0, 0.0, 0.0}, M[3] = {0.0, 0.0, 0.0};

      // particle-particle contacts in partner-id order
      for (int k = 0; k < cnt; k++) {
        const int j = nb[k];
        if (!A[j]) continue;
        const double xj[3] = {X[j], X[n + j], X[2 * n + j]};
        const double Rj = (double)RAD[j];
        const double r = sqrt(sqdist_exact(xi[0], xi[1], xi[2], xj[0], xj[1], xj[2]));
        const double dn = (Ri + Rj) - r;                  // Eq. deltan
        if (!(dn > 0.0)) continue;
        const double dx[3] = {xj[0] - xi[0], xj[1] - xi[1], xj[2] - xi[2]};
        const double nrm[3] = {dx[0] / r, dx[1] / r, dx[2] / r};   // Eq. vecn
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
        const double me = 1.0 / (1.0 / mi + 1.0 / mj);
        double H[3] = {0.0, 0.0, 0.0};
        if ((mold >> k) & 1ull) {
          const int ro = __popcll(mold & ((1ull << k) - 1ull));
          H[0] = Hold[hcomp(P.n, ro, 0)];
          H[1] = Hold[hcomp(P.n, ro, 1)];
          H[2] = Hold[hcomp(P.n, ro, 2)];
        }
        double f[3], nxFt[3], Mr[3];
        law_d(nrm, dn, vij, dw, rwxn, Re, me, Mt.Ye_pp, Mt.Ge_pp, Mt.ceta_pp, Mt.mu_pp, Mt.mur_pp, P.rolling,
              lin ? lin_pp : nullptr, P.dt, H, !init, f, nxFt, Mr);
        for (int d = 0; d < 3; d++) {
          F[d] += f[d];
          M[d] += Ri * nxFt[d] + Mr[d];
        }
        st.touch++;
        st.max_ovl = fmaxf(st.max_ovl, (float)(dn / fmin(Ri, Rj)));
        if (rank < kHistStride) {
          Hnew[hcomp(P.n, rank, 0)] = H[0];
          Hnew[hcomp(P.n, rank, 1)] = H[1];
          Hnew[hcomp(P.n, rank, 2)] = H[2];
          mnew |= 1ull << k;
          rank++;
        } else {
          st.status |= kStCapacity;
        }
      }

      // particle-wall contacts (Sec. 2.1 last paragraph; walls move per Sec. 3.6)
      const double t_now = (double)C->step * P.dt;
      for (int k = 0; k < n_walls; k++) {
        if (!((won >> k) & 1u)) continue;
        const WallDev Wl = wall_at(WLs[k], t_now);
        double nrm[3], dn, ps[3];
        if (!wall_geom_d(Wl, xi, Ri, nrm, &dn, ps)) continue;
        const double arm[3] = {ps[0] - Wl.c[0], ps[1] - Wl.c[1], ps[2] - Wl.c[2]};
        double Vw[3];
        cross3d(Wl.Om, arm, Vw);
        for (int d = 0; d < 3; d++) Vw[d] += Wl.V[d];
        const int bit = kMaxNbr + k;
        double H[3] = {0.0, 0.0, 0.0};
        if ((mold >> bit) & 1ull) {
          const int ro = __popcll(mold & ((1ull << bit) - 1ull));
          H[0] = Hold[hcomp(P.n, ro, 0)];
          H[1] = Hold[hcomp(P.n, ro, 1)];
          H[2] = Hold[hcomp(P.n, ro, 2)];
        }
        double rw[3], rwxn[3], vij[3], dw[3], rdw[3], vom[3];
        for (int d = 0; d < 3; d++) rw[d] = Ri * wi[d];
        cross3d(rw, nrm, rwxn);
        for (int d = 0; d < 3; d++) {
          vij[d] = (vi[d] - Vw[d]) + rwxn[d];
          dw[d] = wi[d] - Wl.Om[d];
          rdw[d] = Ri * dw[d];
        }
        cross3d(rdw, nrm, vom);   // V_omega against the wall: R_i (w_i - Omega) x n
        double f[3], nxFt[3], Mr[3];
        law_d(nrm, dn, vij, dw, vom, Ri, mi, Mt.Ye_pw, Mt.Ge_pw, Mt.ceta_pw, Mt.mu_pw, Mt.mur_pw, P.rolling,
              lin ? lin_pw : nullptr, P.dt, H, !init, f, nxFt, Mr);
        for (int d = 0; d < 3; d++) {
          F[d] += f[d];
          M[d] += Ri * nxFt[d] + Mr[d];
        }
        st.max_ovl = fmaxf(st.max_ovl, (float)(dn / Ri));
        st.wtouch++;
        if (rank < kHistStride) {
          Hnew[hcomp(P.n, rank, 0)] = H[0];
          Hnew[hcomp(P.n, rank, 1)] = H[1];
          Hnew[hcomp(P.n, rank, 2)] = H[2];
          mnew |= 1ull << bit;
          rank++;
        } else {
          st.status |= kStCapacity;
        }
      }
      P.mask[hc ^ 1][i] = mnew;

      // velocity Verlet (Eqs. main1, main2, newvv, halfstep), or explicit Euler (Eq.
      // integ_EE: the state read here is x^n, v^n, and becomes x^{n+1} = x^n + v^n dt,
      // v^{n+1} = v^n + a^n dt)
      double xn[3], vn[3], wn[3];
      const double h = P.half_dt;
      for (int d = 0; d < 3; d++) {
        const double a = F[d] / mi + P.g[d];
        const double al = M[d] / Ii;
        double vf = vi[d], wf = wi[d];
        if (!init && P.integrator == 0) {
          vf = vf + a * h;
          wf = wf + al * h;
        }
        if (last) {
          P.out_v[d * n + i] = vf;
          P.out_w[d * n + i] = wf;
          P.out_F[d * n + i] = F[d];
          P.out_M[d * n + i] = M[d];
        }
        if (P.integrator == 0) {
          vn[d] = vf + a * h;
          wn[d] = wf + al * h;
          xn[d] = xi[d] + vn[d] * P.dt;
        } else {
          xn[d] = xi[d] + vi[d] * P.dt;
          vn[d] = vi[d] + a * P.dt;
          wn[d] = wi[d] + al * P.dt;
        }
        Xo[d * n + i] = xn[d];
        Vo[d * n + i] = vn[d];
        Wo[d * n + i] = wn[d];
      }
      const bool alive = !below_sink(xn[2], P.z_sink_key);
      P.act[nxt][i] = alive ? 1 : 0;
      if (!(finite_d(xn[0]) && finite_d(xn[1]) && finite_d(xn[2]) && finite_d(vn[0]) && finite_d(vn[1]) &&
            finite_d(vn[2])))
        st.status |= kStNonfinite;
      if (alive) {
        st.active++;
        const double xr[3] = {P.xref[i], P.xref[n + i], P.xref[2 * n + i]};
        if (P.rebuild_every <= 0 && sqdist_exact(xr[0], xr[1], xr[2], xn[0], xn[1], xn[2]) > P.disp_lim2)
          P.ctl->need_rebuild = 1;
      }
    }
  }
  if (P.max_overlap_ratio > 0.0 && st.max_ovl > (float)P.max_overlap_ratio) st.status |= kStOverlap;
  end_step(st, P.ctl, last);
}

void launch_step_fp64(const Params& P, cudaStream_t s) {
  const int T = P.step_block > 0 ? P.step_block : step_block(P.n, P.sm_count);
  if (P.n_inst > 1)
    k_step_fp64<true><<<(P.n + T - 1) / T, T, 0, s>>>(P);
  else
    k_step_fp64<false><<<(P.n + T - 1) / T, T, 0, s>>>(P);
}

}  // namespace demgb
