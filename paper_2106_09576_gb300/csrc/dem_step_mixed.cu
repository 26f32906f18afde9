// dem_step_mixed.cu -- mixed-precision step kernel: FP32 contact law, FP64 positions,
// velocities, integration and tangential-overlap accumulation.
//
// One thread owns one particle of the cell-sorted order and walks its inner list (the pairs
// of its fine-search list within R_i + R_j + delta, refreshed before any particle moves
// delta / 2).
// FP64 instructions issue at 1/72 of the FP32 rate on this part, so the kernel keeps them
// to the integration (9 FMAs per particle) and the tangential-overlap accumulation
// (3 adds per contact).  Every particle publishes, once per step, a 48-byte FP32 copy of
// itself for its neighbours, {x_hi, x_lo, v, w} (the radius is in its own array, and a
// particle out of the system sits at kFar); the inner-list build and a contact partner
// read it, its own thread starts from it too and reads its FP64 state only for walls and
// integration.
//   - relative positions are exact two-sum differences of the hi + lo pairs, so nearly
//     co-located spheres keep their relative position to ~1e-7;
//   - the normal overlap is (S^2 - r^2) / (S + r) with S^2 - r^2 formed exactly as a
//     double-float (no cancellation at small overlaps);
//   - FP32<->FP64 conversions use integer operations; uniform constants arrive in FP32;
//     the rebuild trigger, the z_sink test and the wall time windows use no FP64 work.
#include "dem_step_common.cuh"

namespace demgb {

// Sends the cache line of p towards L1 (no register holds the data): the step kernels
// issue it for the next slot's partner while the current slot computes.
__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// One particle-wall contact: FP64 geometry, FP32 law, FP64 overlap accumulation.  Few
// particles touch a wall, so this is kept out of line: its FP64 temporaries would
// otherwise set the register budget (and the spills) of the whole kernel.
struct WallOut {
  float F[3], M[3];
  double H[3];
  float ovl;
  int hit;
};

// A particle's FP32 copy unpacked: position as hi + lo, velocity and spin.
struct OwnF {
  float xh[3], xl[3], v[3], w[3];
};

// Geometry of a contact with an axis-aligned plane or cylinder (WallX) in double-float FP32,
// the same quantities as the FP64 form: normal (from the particle towards the wall), overlap
// and the contact point's arm from the rotation origin.  The difference x - p is an exact
// two-sum of the hi + lo pairs; a plane's overlap R - n.(x - p) keeps R - sign s exact near
// contact; a cylinder's overlap rho - (radius - R) is formed as (rho^2 - Q^2) / (rho + Q),
// Q = radius - R, with both squares exact double-floats, as the pair overlap is.  Returns 0
// without contact, 1 with one, 2 if the FP64 form must decide (a particle wider than the
// cylinder).
__device__ __forceinline__ int wall_geom_x(const WallX& X, int kind, const OwnF& own, float R, float* nrm, float* dn,
                                           float* arm) {
  const int a = X.axis;
  const float sg = X.sign;
  float s[3], t[3];
  for (int d = 0; d < 3; d++) df_diff(X.ph[d], X.pl[d], own.xh[d], own.xl[d], s[d], t[d]);   // x - p
  if (kind == 0) {
    const float ov = (R - sg * s[a]) - sg * t[a];
    if (!(ov > 0.0f)) return 0;
    for (int d = 0; d < 3; d++) {
      nrm[d] = d == a ? -sg : 0.0f;
      // p* = x - (n.(x - p)) n: p on the normal's axis, x on the others
      arm[d] = (d == a ? X.ph[d] + X.pl[d] : own.xh[d] + own.xl[d]) - X.c[d];
    }
    *dn = ov;
    return 1;
  }
  const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
  float Ah, Al, pe, p2, e2;
  two_prod(s[b], s[b], Ah, pe);
  Al = pe + (2.0f * s[b] + t[b]) * t[b];
  two_prod(s[c], s[c], p2, pe);
  two_sum(Ah, p2, Ah, e2);
  Al += e2 + pe + (2.0f * s[c] + t[c]) * t[c];
  float Qh, Qe;
  two_sum(X.rh, -R, Qh, Qe);
  const float Ql = Qe + X.rl;
  if (!(Qh > 0.0f)) return 2;
  float Q2, Q2e, Dh, De;
  two_prod(Qh, Qh, Q2, Q2e);
  Q2e += 2.0f * Qh * Ql;
  two_sum(Ah, -Q2, Dh, De);
  const float D = Dh + (De + (Al - Q2e));
  if (!(D > 0.0f)) return 0;
  const float rho = sqrtf(Ah + Al);
  *dn = D / (rho + (Qh + Ql));
  const float ir = 1.0f / rho;
  for (int d = 0; d < 3; d++) {
    const float u = d == a ? 0.0f : (s[d] + t[d]) * ir;
    nrm[d] = u;
    // p* = p + (n.(x - p)) n + radius u: x on the axis, p + radius u across it
    arm[d] = (d == a ? own.xh[d] + own.xl[d] : (X.ph[d] + X.pl[d]) + (X.rh + X.rl) * u) - X.c[d];
  }
  return 1;
}

template <bool kBatch, bool kExt>
__device__ __noinline__ WallOut wall_contact_mixed(const Params* Pp, const InstDev* I, int k, int i, int cur, float Rif,
                                                   float mif, unsigned long long mold, const double* Hold, bool init) {
  const Params& P = *Pp;
  const WallDev& Wl = kBatch ? I->walls[k] : P.walls[k];
  const WallX& Xw = kBatch ? I->wx[k] : P.wx[k];

  const MatF& Mt = kBatch ? I->mf : P.mf;
  WallOut o;
  o.hit = 0;
  // normal, overlap, v_i - V_wall(p*), w_i - Omega and w_i in FP32
  float nf[3], dnf, dv[3], dw[3], wif[3];
  int geo = 2;
  if (Xw.axis >= 0) {
    // the particle's FP32 copy, read again here (rare) rather than kept live by the caller
    const float4* rd = P.render[cur] + 3 * (size_t)i;
    const float4 q0 = rd[0], q1 = rd[1], q2 = rd[2];
    const OwnF own = {{q0.x, q0.y, q0.z}, {q0.w, q1.x, q1.y}, {q1.z, q1.w, q2.x}, {q2.y, q2.z, q2.w}};
    float arm[3];
    geo = wall_geom_x(Xw, Wl.kind, own, Rif, nf, &dnf, arm);
    if (geo == 0) return o;
    if (geo == 1) {
      const float Vw[3] = {Xw.Om[1] * arm[2] - Xw.Om[2] * arm[1] + Xw.V[0],
                           Xw.Om[2] * arm[0] - Xw.Om[0] * arm[2] + Xw.V[1],
                           Xw.Om[0] * arm[1] - Xw.Om[1] * arm[0] + Xw.V[2]};
      for (int d = 0; d < 3; d++) {
        dv[d] = own.v[d] - Vw[d];
        dw[d] = own.w[d] - Xw.Om[d];
        wif[d] = own.w[d];
      }
    }
  }
  if (geo == 2) {
    // any other wall: FP64 geometry
    const int n = P.n;
    double xi[3] = {P.x[cur][i], P.x[cur][n + i], P.x[cur][2 * n + i]};
    if (kExt && Wl.translates) {   // a translating wall is handled in its own frame: x - V t
      const double tw = (double)P.ctl->step * P.dt;
      for (int d = 0; d < 3; d++) xi[d] = xi[d] - Wl.V[d] * tw;
    }
    double nrmd[3], dnd, ps[3];   // ps in the wall's frame: p* - c is the same in both frames
    if (!wall_geom_d(Wl, xi, (double)Rif, nrmd, &dnd, ps)) return o;
    const double arm[3] = {ps[0] - Wl.c[0], ps[1] - Wl.c[1], ps[2] - Wl.c[2]};
    double Vw[3];
    cross3d(Wl.Om, arm, Vw);
    for (int d = 0; d < 3; d++) Vw[d] += Wl.V[d];
    for (int d = 0; d < 3; d++) nf[d] = (float)nrmd[d];
    dnf = (float)dnd;
    // v_i - V_wall(p*) and w_i - Omega as exact double-float differences
    for (int d = 0; d < 3; d++) {
      const double vi = P.v[cur][d * n + i], wi = P.w[cur][d * n + i];
      float ah, al, bh, bl, s1, t1;
      split_df(vi, ah, al);
      split_df(Vw[d], bh, bl);
      df_diff(bh, bl, ah, al, s1, t1);
      dv[d] = s1 + t1;
      split_df(wi, ah, al);
      split_df(Wl.Om[d], bh, bl);
      df_diff(bh, bl, ah, al, s1, t1);
      dw[d] = s1 + t1;
      wif[d] = d2f_int(wi);
    }
  }
  const int bit = kMaxNbr + k;
  double H[3] = {0.0, 0.0, 0.0};
  if ((mold >> bit) & 1ull) {
    const int ro = __popcll(mold & ((1ull << bit) - 1ull));
    H[0] = Hold[hcomp(P.n, ro, 0)];
    H[1] = Hold[hcomp(P.n, ro, 1)];
    H[2] = Hold[hcomp(P.n, ro, 2)];
  }
  const float rw[3] = {Rif * wif[0], Rif * wif[1], Rif * wif[2]};
  const float vij[3] = {dv[0] + (rw[1] * nf[2] - rw[2] * nf[1]), dv[1] + (rw[2] * nf[0] - rw[0] * nf[2]),
                        dv[2] + (rw[0] * nf[1] - rw[1] * nf[0])};
  // V_omega against the wall (viscous rolling): R_i (w_i - Omega) x n
  const float rdw[3] = {Rif * dw[0], Rif * dw[1], Rif * dw[2]};
  const float vom[3] = {rdw[1] * nf[2] - rdw[2] * nf[1], rdw[2] * nf[0] - rdw[0] * nf[2],
                        rdw[0] * nf[1] - rdw[1] * nf[0]};
  const float lin[2] = {P.f_lin_V, Mt.lin_den_pw};
  float F[3] = {0.f, 0.f, 0.f}, M[3] = {0.f, 0.f, 0.f};
  law_f<kExt>(nf, dnf, vij, dw, vom, Rif, mif, Mt.Ye_pw, Mt.Ge_pw, Mt.ceta_pw, Mt.mu_pw, Mt.mur_pw, P.rolling,
        P.contact_model == 1 ? lin : nullptr, P.f_dt, H, !init, Rif, F, M);
  for (int d = 0; d < 3; d++) {
    o.F[d] = F[d];
    o.M[d] = M[d];
    o.H[d] = H[d];
  }
  o.ovl = dnf / Rif;
  o.hit = 1;
  return o;
}

template <bool kBatch, bool kExt>
__global__ void __launch_bounds__(kStepBlock, 6) k_step_mixed(const __grid_constant__ Params P) {
  const Control* C = P.ctl;
  const int cur = C->cur, nxt = cur ^ 1, hc = C->hc;
  const bool init = C->init != 0, last = C->last != 0;
  const unsigned wall_on = C->wall_on;
  const int n = P.n, nact = C->n_act_sorted;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  StepStats st = {0u, 0u, 0u, 0.0f, 0u};
  const double* X = P.x[cur];
  const double* V = P.v[cur];
  const double* W = P.w[cur];
  const float4* RD = P.render[cur];
  const float* RAD = P.rad[C->sbuf];
  float4* RDo = P.render[nxt];

  if (last && i >= nact && i < n) {
    for (int d = 0; d < 3; d++) {   // out of the system: frozen in both buffers
      P.out_v[d * n + i] = V[d * n + i];
      P.out_w[d * n + i] = W[d * n + i];
      P.out_F[d * n + i] = 0.0;
      P.out_M[d * n + i] = 0.0;
    }
  }
  if (i < nact) {
    const float4 o0 = RD[3 * (size_t)i];
    if (o0.x == kFar) {
      for (int d = 0; d < 3; d++) {
        const double xv = X[d * n + i], vv = V[d * n + i], wv = W[d * n + i];
        P.x[nxt][d * n + i] = xv;
        P.v[nxt][d * n + i] = vv;
        P.w[nxt][d * n + i] = wv;
        if (last) {
          P.out_v[d * n + i] = vv;
          P.out_w[d * n + i] = wv;
          P.out_F[d * n + i] = 0.0;
          P.out_M[d * n + i] = 0.0;
        }
      }
      P.act[nxt][i] = 0;
      P.mask[hc ^ 1][i] = 0ull;
      for (int k = 0; k < 3; k++) RDo[3 * (size_t)i + k] = RD[3 * (size_t)i + k];
    } else {
      const float4 o1 = RD[3 * (size_t)i + 1];
      const float hx[3] = {o0.x, o0.y, o0.z}, lx[3] = {o0.w, o1.x, o1.y};
      const float Rif = RAD[i];
      // materials and walls: the context's, or those of the particle's instance in a batch
      const InstDev* I = kBatch ? P.itab + P.inst[C->sbuf][i] : nullptr;
      const MatF& Mt = kBatch ? I->mf : P.mf;
      // ---------------- particle-particle contacts
      // The inner list holds the slots of the fine-search list whose partner was within
      // R_i + R_j + delta when it was built; no particle has moved delta / 2 since, so it
      // holds every touching pair, in partner-id order (a serial pair loop's order).
      const uint8_t* irow = P.inner + (size_t)i * kInnerMax;
      const int* jrow = P.inner_j + (size_t)i * kInnerMax;
      const int icnt = P.inner_cnt[i];
      const float4 o2 = RD[3 * (size_t)i + 2];
      const float vif[3] = {o1.z, o1.w, o2.x}, wif[3] = {o2.y, o2.z, o2.w};
      const unsigned long long mold = P.mask[hc][i];
      const double* Hold = P.hist[hc] + (size_t)i;
      double* Hnew = P.hist[hc ^ 1] + (size_t)i;
      const float mif = P.f_density * (4.0f / 3.0f) * 3.14159265358979f * Rif * Rif * Rif;
      const float dtf = P.f_dt;
      float Ff[3] = {0.f, 0.f, 0.f}, Mf[3] = {0.f, 0.f, 0.f};
      unsigned long long mnew = 0ull;
      int rank = 0;

      // every load of a candidate is issued before any branch; the first row entry is read
      // without waiting for the count (it exists for every particle; unused if the row is
      // empty), each next one with the prefetch of its partner
      int kc = irow[0], jc = jrow[0];
      for (int slot = 0; slot < icnt; slot++) {
        const int k = kc;
        const int j = jc;
        const float4* rj = RD + 3 * (size_t)j;
        const float4 r0 = rj[0], r1 = rj[1], r2 = rj[2];
        const float Rjf = RAD[j];
        double H[3] = {0.0, 0.0, 0.0};
        if ((mold >> k) & 1ull) {
          const int ro = __popcll(mold & ((1ull << k) - 1ull));
          H[0] = Hold[hcomp(P.n, ro, 0)];
          H[1] = Hold[hcomp(P.n, ro, 1)];
          H[2] = Hold[hcomp(P.n, ro, 2)];
        }
        // the next slot's partner copy, radius and overlap towards L1 (its row entries are
        // in the sector just read)
        if (slot + 1 < icnt) {
          const int k1 = irow[slot + 1], j1 = jrow[slot + 1];
          kc = k1;
          jc = j1;
          const char* r1p = reinterpret_cast<const char*>(RD + 3 * (size_t)j1);
          prefetch_l1(r1p);
          prefetch_l1(r1p + 32);
          prefetch_l1(RAD + j1);
          if ((mold >> k1) & 1ull) {
            const int ro1 = __popcll(mold & ((1ull << k1) - 1ull));
            prefetch_l1(Hold + hcomp(P.n, ro1, 0));
            prefetch_l1(Hold + hcomp(P.n, ro1, 1));
            prefetch_l1(Hold + hcomp(P.n, ro1, 2));
          }
        }
        if (r0.x == kFar) continue;                    // partner out of the system
        float s[3], t[3], dxf[3];
        df_diff(hx[0], lx[0], r0.x, r0.w, s[0], t[0]);
        df_diff(hx[1], lx[1], r0.y, r1.x, s[1], t[1]);
        df_diff(hx[2], lx[2], r0.z, r1.y, s[2], t[2]);
        for (int d = 0; d < 3; d++) dxf[d] = s[d] + t[d];
        const float S = Rif + Rjf;
        // S^2 - r^2 as an exact double-float
        float p2, pe, e, Ah, Al;
        two_prod(s[0], s[0], Ah, pe);
        Al = pe + (2.0f * s[0] + t[0]) * t[0];
        two_prod(s[1], s[1], p2, pe);
        two_sum(Ah, p2, Ah, e);
        Al += e + pe + (2.0f * s[1] + t[1]) * t[1];
        two_prod(s[2], s[2], p2, pe);
        two_sum(Ah, p2, Ah, e);
        Al += e + pe + (2.0f * s[2] + t[2]) * t[2];
        float Sh, Sl, P2, P2e, Dh, De;
        two_sum(Rif, Rjf, Sh, Sl);
        two_prod(Sh, Sh, P2, P2e);
        P2e += 2.0f * Sh * Sl;
        two_sum(P2, -Ah, Dh, De);
        const float D = Dh + (De + (P2e - Al));
        if (!(D > 0.0f)) continue;
        const float r = sqrtf(Ah + Al);
        const float dn = D / (Sh + r);                   // Eq. deltan without cancellation
        const float ir = 1.0f / r;
        const float nrm[3] = {dxf[0] * ir, dxf[1] * ir, dxf[2] * ir};   // Eq. vecn
        const float wj[3] = {r2.y, r2.z, r2.w};
        const float dv[3] = {vif[0] - r1.z, vif[1] - r1.w, vif[2] - r2.x};
        const float dw[3] = {wif[0] - wj[0], wif[1] - wj[1], wif[2] - wj[2]};
        // R_i w_i + R_j w_j rounded identically on both sides of the pair (no contraction),
        // so the two sides' tangential overlaps stay exact opposites and a contact search,
        // which restores one side's overlap from the other's, leaves the trajectory unchanged
        float rw[3];
        for (int d = 0; d < 3; d++) rw[d] = __fadd_rn(__fmul_rn(Rif, wif[d]), __fmul_rn(Rjf, wj[d]));
        // (R_i w_i + R_j w_j) x n: part of v_ij, and V_omega of the viscous rolling model
        const float rwxn[3] = {rw[1] * nrm[2] - rw[2] * nrm[1], rw[2] * nrm[0] - rw[0] * nrm[2],
                               rw[0] * nrm[1] - rw[1] * nrm[0]};
        const float vij[3] = {dv[0] + rwxn[0], dv[1] + rwxn[1], dv[2] + rwxn[2]};
        const float Re = Rif * Rjf / S;
        const float mj = P.f_density * (4.0f / 3.0f) * 3.14159265358979f * Rjf * Rjf * Rjf;
        const float me = mif * mj / (mif + mj);
        const float lin[2] = {P.f_lin_V, Mt.lin_den_pp};
        law_f<kExt>(nrm, dn, vij, dw, rwxn, Re, me, Mt.Ye_pp, Mt.Ge_pp, Mt.ceta_pp, Mt.mu_pp, Mt.mur_pp, P.rolling,
              P.contact_model == 1 ? lin : nullptr, dtf, H, !init, Rif, Ff, Mf);
        st.touch++;
        st.max_ovl = fmaxf(st.max_ovl, dn / fminf(Rif, Rjf));
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

      // ---------------- particle-wall contacts (FP32 prefilter, then out of line)
      const float xf[3] = {hx[0] + lx[0], hx[1] + lx[1], hx[2] + lx[2]};
      const WallDev* WLs = kBatch ? I->walls : P.walls;
      const WallF* WFs = kBatch ? I->wf : P.wf;
      const int n_walls = kBatch ? I->n_walls : P.n_walls;
      unsigned won = wall_on;
      if (kBatch) {
        won = 0u;
        const double t = (double)C->step * P.dt;
        for (int k = 0; k < n_walls; k++)
          if (t >= WLs[k].t_on && t < WLs[k].t_off) won |= 1u << k;
      }
      const float t_now = (float)C->step * P.f_dt;
      for (int k = 0; k < n_walls; k++) {
        if (!((won >> k) & 1u)) continue;
        // the particle seen from a translating wall's frame (v = 0 for other walls)
        if (kExt) {
          const float* wv = kBatch ? I->wf_v[k] : P.wf_v[k];
          const float xs[3] = {xf[0] - wv[0] * t_now, xf[1] - wv[1] * t_now, xf[2] - wv[2] * t_now};
          if (!wall_maybe_f(WLs[k].kind, WFs[k], xs, Rif, P.wall_margin)) continue;
        } else if (!wall_maybe_f(WLs[k].kind, WFs[k], xf, Rif, P.wall_margin)) {
          continue;
        }
        const WallOut o = wall_contact_mixed<kBatch, kExt>(&P, I, k, i, cur, Rif, mif, mold, Hold, init);
        if (!o.hit) continue;
        for (int d = 0; d < 3; d++) {
          Ff[d] += o.F[d];
          Mf[d] += o.M[d];
        }
        st.max_ovl = fmaxf(st.max_ovl, o.ovl);
        st.wtouch++;
        if (rank < kHistStride) {
          Hnew[hcomp(P.n, rank, 0)] = o.H[0];
          Hnew[hcomp(P.n, rank, 1)] = o.H[1];
          Hnew[hcomp(P.n, rank, 2)] = o.H[2];
          mnew |= 1ull << (kMaxNbr + k);
          rank++;
        } else {
          st.status |= kStCapacity;
        }
      }
      P.mask[hc ^ 1][i] = mnew;

      // ---------------- velocity Verlet in FP64 with FP32 accelerations (Eqs. main1, main2),
      // or explicit Euler (Eq. integ_EE: x^{n+1} = x^n + v^n dt, v^{n+1} = v^n + a^n dt)
      const float inv_m = 1.0f / mif;
      const float inv_I = 1.0f / (0.4f * mif * Rif * Rif);
      double xn[3], vn[3], wn[3];
      for (int d = 0; d < 3; d++) {
        // the own FP64 state, read only now: fewer registers live through the contacts
        const double xi = X[d * n + i], vi = V[d * n + i], wi = W[d * n + i];
        const double a = f2d_int(Ff[d] * inv_m + P.f_g[d]);
        const double al = f2d_int(Mf[d] * inv_I);
        const bool euler = kExt && P.integrator == 1;
        if (init && !euler) {
          vn[d] = fma(a, P.half_dt, vi);
          wn[d] = fma(al, P.half_dt, wi);
        } else {
          vn[d] = fma(a, P.dt, vi);
          wn[d] = fma(al, P.dt, wi);
        }
        if (last) {
          P.out_v[d * n + i] = (init || euler) ? vi : fma(a, P.half_dt, vi);
          P.out_w[d * n + i] = (init || euler) ? wi : fma(al, P.half_dt, wi);
          P.out_F[d * n + i] = f2d_int(Ff[d]);
          P.out_M[d * n + i] = f2d_int(Mf[d]);
        }
        xn[d] = fma(euler ? vi : vn[d], P.dt, xi);
        P.x[nxt][d * n + i] = xn[d];
        P.v[nxt][d * n + i] = vn[d];
        P.w[nxt][d * n + i] = wn[d];
      }
      const bool alive = !below_sink(xn[2], P.z_sink_key);
      P.act[nxt][i] = alive ? 1 : 0;
      float hn[3], ln[3];
      for (int d = 0; d < 3; d++) split_df(xn[d], hn[d], ln[d]);
      write_render(RDo + 3 * (size_t)i, hn, ln, vn, wn, alive);
      if (!(finite_d(xn[0]) && finite_d(xn[1]) && finite_d(xn[2]) && finite_d(vn[0]) && finite_d(vn[1]) &&
            finite_d(vn[2])))
        st.status |= kStNonfinite;
      if (alive) {
        st.active++;
        // triggers on the hi + lo pairs, without FP64 arithmetic: the inner list is due when
        // |x^{n+1} - x_in| > delta / 2; the contact search (as the method states it) when
        // |x^{n+1} - x_ref| > skin / 2, which is tested only when |x^{n+1} - x_in| plus the
        // stored |x_in - x_ref| come near skin / 2 (below, it cannot hold)
        const float dm = moved_since_inner(P.xin, n, i, hn, ln);
        if (dm * dm > P.f_inner_lim2) P.ctl->need_inner = 1;
        if (P.rebuild_every <= 0 && dm + P.xin[3 * (size_t)n + i] > P.f_disp_lim * (1.0f - 1e-5f)) {
          const float* xs = reinterpret_cast<const float*>(P.xref);
          float e2 = 0.f;
          for (int d = 0; d < 3; d++) {
            float s1, t1;
            df_diff(xs[d * n + i], xs[(3 + d) * n + i], hn[d], ln[d], s1, t1);
            const float u = s1 + t1;
            e2 += u * u;
          }
          if (e2 > P.f_disp_lim2) P.ctl->need_rebuild = 1;
        }
      }
    }
  }
  if (P.max_overlap_ratio > 0.0 && st.max_ovl > (float)P.max_overlap_ratio) st.status |= kStOverlap;
  end_step(st, P.ctl, last);
}

// ====================================================================== one evaluation per pair
// A touching pair is evaluated once, by its partner of smaller id (the owner), with the
// law and operations of the kernel above: the two sides of a pair compute exact opposites
// there (Sec. 2.1: the pair force and its reaction; Eq. torque_t, with the same n x F_t on
// both sides; Table rolling_torque, w_ji = -w_ij), so the owner's numbers give the
// partner's contribution exactly.  The step is two kernels:
//   k_pair_mixed  per owner: its owned inner slots (partners of larger id, in id order)
//                 and its walls; the owner's own sum into upart, the partner's reaction
//                 -F, R_j n x F_t - M_r into the partner's record rec[m][j] (m: the
//                 owner's slot in the partner's inner list), zeros for a pair that does
//                 not touch; the owner keeps the pair's tangential overlap;
//   k_int_mixed   per particle: the records of its leading slots (partners that own the
//                 pair, in id order), plus its own sum, then integration as above.
// Every sum has a fixed order given by the touching pairs alone (records first, then the
// owner's pairs in id order, then walls), so a trajectory does not depend on when the
// lists are rebuilt; no float atomics.
__device__ __forceinline__ void put_rec(const Params& P, int m, int j, const float* f, const float* t) {
  float4* r = P.rec + 2 * ((size_t)m * P.n + j);
  r[0] = make_float4(f[0], f[1], f[2], t[0]);
  r[1] = make_float4(t[1], t[2], 0.0f, 0.0f);
}

template <bool kBatch, bool kExt>
__global__ void __launch_bounds__(kStepBlock, 6) k_pair_mixed(const __grid_constant__ Params P) {
  const Control* C = P.ctl;
  const int cur = C->cur, hc = C->hc;
  const bool init = C->init != 0, last = C->last != 0;
  const unsigned wall_on = C->wall_on;
  const int n = P.n, nact = C->n_act_sorted;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  StepStats st = {0u, 0u, 0u, 0.0f, 0u};
  // read-only in this kernel: the compiler may issue these loads ahead of the stores
  const float4* __restrict__ RD = P.render[cur];
  const float* __restrict__ RAD = P.rad[C->sbuf];
  if (i < nact) {
    const int icnt = P.inner_cnt[i], ilo = P.inner_lo[i];
    const int nown = icnt - ilo;
    const int2* __restrict__ ps = P.pslot + i;   // entry t at ps[t * n]: slot-major
    // the first two owned-slot entries are read with the own data, without waiting for the
    // counts (entries 0 and 1 exist for every particle; those beyond the owned count are
    // never used); each later one during the arithmetic of the slot two before it
    int2 e = __ldg(ps);
    int2 e1 = __ldg(ps + (size_t)n);
    const float4 o0 = __ldg(RD + 3 * (size_t)i);
    const float zero[3] = {0.f, 0.f, 0.f};
    float Ff[3] = {0.f, 0.f, 0.f}, Mf[3] = {0.f, 0.f, 0.f};
    if (o0.x == kFar) {
      // out of the system: its pairs exert nothing, and its partners' records say so
      for (int t = 0; t < nown; t++) {
        const int2 f = __ldg(ps + (size_t)t * n);
        const int m = (f.y >> 8) & 0xFF;
        if (m != 255) put_rec(P, m, f.x, zero, zero);
      }
      P.mask[hc ^ 1][i] = 0ull;
    } else {
      const float4 o1 = __ldg(RD + 3 * (size_t)i + 1), o2 = __ldg(RD + 3 * (size_t)i + 2);
      const float hx[3] = {o0.x, o0.y, o0.z}, lx[3] = {o0.w, o1.x, o1.y};
      const float Rif = __ldg(RAD + i);
      const InstDev* I = kBatch ? P.itab + P.inst[C->sbuf][i] : nullptr;
      const MatF& Mt = kBatch ? I->mf : P.mf;
      const float vif[3] = {o1.z, o1.w, o2.x}, wif[3] = {o2.y, o2.z, o2.w};
      const unsigned long long mold = __ldg(P.mask[hc] + i);
      const double* __restrict__ Hold = P.hist[hc] + (size_t)i;
      double* Hnew = P.hist[hc ^ 1] + (size_t)i;
      const float mif = P.f_density * (4.0f / 3.0f) * 3.14159265358979f * Rif * Rif * Rif;
      const float dtf = P.f_dt;
      unsigned long long mnew = 0ull;
      int rank = 0;
      for (int t = 0; t < nown; t++) {
        const int j = e.x;
        const int k = e.y & 0xFF;
        const int m = (e.y >> 8) & 0xFF;
        const float4* rj = RD + 3 * (size_t)j;
        const float4 r0 = __ldg(rj), r1 = __ldg(rj + 1), r2 = __ldg(rj + 2);
        const float rj_R = __ldg(RAD + j);
        double H[3] = {0.0, 0.0, 0.0};
        if ((mold >> k) & 1ull) {
          const int ro = __popcll(mold & ((1ull << k) - 1ull));
          H[0] = __ldg(Hold + hcomp(P.n, ro, 0));
          H[1] = __ldg(Hold + hcomp(P.n, ro, 1));
          H[2] = __ldg(Hold + hcomp(P.n, ro, 2));
        }
        // the next slot's partner copy, radius and overlap are sent towards L1 now, so that
        // its loads hit there; the entry after it is fetched into a register
        if (t + 1 < nown) {
          const int j1 = e1.x, k1 = e1.y & 0xFF;
          const char* r1p = reinterpret_cast<const char*>(RD + 3 * (size_t)j1);
          prefetch_l1(r1p);
          prefetch_l1(r1p + 32);
          prefetch_l1(RAD + j1);
          if ((mold >> k1) & 1ull) {
            const int ro1 = __popcll(mold & ((1ull << k1) - 1ull));
            prefetch_l1(Hold + hcomp(P.n, ro1, 0));
            prefetch_l1(Hold + hcomp(P.n, ro1, 1));
            prefetch_l1(Hold + hcomp(P.n, ro1, 2));
          }
          e = e1;
          if (t + 2 < nown) e1 = __ldg(ps + (size_t)(t + 2) * n);
        }
        float rf[3] = {0.f, 0.f, 0.f}, rm[3] = {0.f, 0.f, 0.f};
        bool touch = false;
        float Rjf = 0.f, D = 0.f, Sh = 0.f, Ah = 0.f, Al = 0.f;
        float s3[3], t3[3];
        if (r0.x != kFar) {                              // partner in the system
          Rjf = rj_R;
          df_diff(hx[0], lx[0], r0.x, r0.w, s3[0], t3[0]);
          df_diff(hx[1], lx[1], r0.y, r1.x, s3[1], t3[1]);
          df_diff(hx[2], lx[2], r0.z, r1.y, s3[2], t3[2]);
          // S^2 - r^2 as an exact double-float
          float p2, pe, e2;
          two_prod(s3[0], s3[0], Ah, pe);
          Al = pe + (2.0f * s3[0] + t3[0]) * t3[0];
          two_prod(s3[1], s3[1], p2, pe);
          two_sum(Ah, p2, Ah, e2);
          Al += e2 + pe + (2.0f * s3[1] + t3[1]) * t3[1];
          two_prod(s3[2], s3[2], p2, pe);
          two_sum(Ah, p2, Ah, e2);
          Al += e2 + pe + (2.0f * s3[2] + t3[2]) * t3[2];
          float Sl, P2, P2e, Dh, De;
          two_sum(Rif, Rjf, Sh, Sl);
          two_prod(Sh, Sh, P2, P2e);
          P2e += 2.0f * Sh * Sl;
          two_sum(P2, -Ah, Dh, De);
          D = Dh + (De + (P2e - Al));
          touch = D > 0.0f;
        }
        if (touch) {
          float dxf[3];
          for (int d = 0; d < 3; d++) dxf[d] = s3[d] + t3[d];
          const float S = Rif + Rjf;
          const float r = sqrtf(Ah + Al);
          const float dn = D / (Sh + r);                   // Eq. deltan without cancellation
          const float ir = 1.0f / r;
          const float nrm[3] = {dxf[0] * ir, dxf[1] * ir, dxf[2] * ir};   // Eq. vecn
          const float wj[3] = {r2.y, r2.z, r2.w};
          const float dv[3] = {vif[0] - r1.z, vif[1] - r1.w, vif[2] - r2.x};
          const float dw[3] = {wif[0] - wj[0], wif[1] - wj[1], wif[2] - wj[2]};
          float rw[3];
          for (int d = 0; d < 3; d++) rw[d] = __fadd_rn(__fmul_rn(Rif, wif[d]), __fmul_rn(Rjf, wj[d]));
          const float rwxn[3] = {rw[1] * nrm[2] - rw[2] * nrm[1], rw[2] * nrm[0] - rw[0] * nrm[2],
                                 rw[0] * nrm[1] - rw[1] * nrm[0]};
          const float vij[3] = {dv[0] + rwxn[0], dv[1] + rwxn[1], dv[2] + rwxn[2]};
          const float Re = Rif * Rjf / S;
          const float mj = P.f_density * (4.0f / 3.0f) * 3.14159265358979f * Rjf * Rjf * Rjf;
          const float me = mif * mj / (mif + mj);
          const float lin[2] = {P.f_lin_V, Mt.lin_den_pp};
          float Fp[3], nxFt[3], Mr[3];
          law_pieces_f<kExt>(nrm, dn, vij, dw, rwxn, Re, me, Mt.Ye_pp, Mt.Ge_pp, Mt.ceta_pp, Mt.mu_pp, Mt.mur_pp,
                             P.rolling, P.contact_model == 1 ? lin : nullptr, dtf, H, !init, Fp, nxFt, Mr);
          for (int d = 0; d < 3; d++) {
            Ff[d] += Fp[d];
            Mf[d] += Rif * nxFt[d] + Mr[d];
            rf[d] = -Fp[d];
            rm[d] = Rjf * nxFt[d] - Mr[d];
          }
          st.touch += 2u;
          st.max_ovl = fmaxf(st.max_ovl, dn / fminf(Rif, Rjf));
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
        if (m != 255) put_rec(P, m, j, rf, rm);
      }

      // ---------------- particle-wall contacts (FP32 prefilter, then out of line)
      const float xf[3] = {hx[0] + lx[0], hx[1] + lx[1], hx[2] + lx[2]};
      const WallDev* WLs = kBatch ? I->walls : P.walls;
      const WallF* WFs = kBatch ? I->wf : P.wf;
      const int n_walls = kBatch ? I->n_walls : P.n_walls;
      unsigned won = wall_on;
      if (kBatch) {
        won = 0u;
        const double t = (double)C->step * P.dt;
        for (int k = 0; k < n_walls; k++)
          if (t >= WLs[k].t_on && t < WLs[k].t_off) won |= 1u << k;
      }
      const float t_now = (float)C->step * P.f_dt;
      for (int k = 0; k < n_walls; k++) {
        if (!((won >> k) & 1u)) continue;
        if (kExt) {
          const float* wv = kBatch ? I->wf_v[k] : P.wf_v[k];
          const float xs[3] = {xf[0] - wv[0] * t_now, xf[1] - wv[1] * t_now, xf[2] - wv[2] * t_now};
          if (!wall_maybe_f(WLs[k].kind, WFs[k], xs, Rif, P.wall_margin)) continue;
        } else if (!wall_maybe_f(WLs[k].kind, WFs[k], xf, Rif, P.wall_margin)) {
          continue;
        }
        const WallOut o = wall_contact_mixed<kBatch, kExt>(&P, I, k, i, cur, Rif, mif, mold, Hold, init);
        if (!o.hit) continue;
        for (int d = 0; d < 3; d++) {
          Ff[d] += o.F[d];
          Mf[d] += o.M[d];
        }
        st.max_ovl = fmaxf(st.max_ovl, o.ovl);
        st.wtouch++;
        if (rank < kHistStride) {
          Hnew[hcomp(P.n, rank, 0)] = o.H[0];
          Hnew[hcomp(P.n, rank, 1)] = o.H[1];
          Hnew[hcomp(P.n, rank, 2)] = o.H[2];
          mnew |= 1ull << (kMaxNbr + k);
          rank++;
        } else {
          st.status |= kStCapacity;
        }
      }
      P.mask[hc ^ 1][i] = mnew;
    }
    // six planes of n floats: a warp writes 128 contiguous bytes per plane
    for (int d = 0; d < 3; d++) {
      P.upart[(size_t)d * n + i] = Ff[d];
      P.upart[(size_t)(3 + d) * n + i] = Mf[d];
    }
  }
  if (P.max_overlap_ratio > 0.0 && st.max_ovl > (float)P.max_overlap_ratio) st.status |= kStOverlap;
  end_step(st, P.ctl, last, false);
}

constexpr int kIntBlock = 256;

template <bool kExt>
__global__ void __launch_bounds__(kIntBlock, 4) k_int_mixed(const __grid_constant__ Params P) {
  const Control* C = P.ctl;
  const int cur = C->cur, nxt = cur ^ 1, hc = C->hc;
  const bool init = C->init != 0, last = C->last != 0;
  const int n = P.n, nact = C->n_act_sorted;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  StepStats st = {0u, 0u, 0u, 0.0f, 0u};
  const double* X = P.x[cur];
  const double* V = P.v[cur];
  const double* W = P.w[cur];
  const float4* RD = P.render[cur];
  float4* RDo = P.render[nxt];

  if (last && i >= nact && i < n) {
    for (int d = 0; d < 3; d++) {   // out of the system: frozen in both buffers
      P.out_v[d * n + i] = V[d * n + i];
      P.out_w[d * n + i] = W[d * n + i];
      P.out_F[d * n + i] = 0.0;
      P.out_M[d * n + i] = 0.0;
    }
  }
  if (i < nact) {
    // the in-system flag and the radius from their own arrays: 5 bytes instead of the
    // FP32 copy's first vector
    if (P.act[cur][i] == 0) {
      for (int d = 0; d < 3; d++) {
        const double xv = X[d * n + i], vv = V[d * n + i], wv = W[d * n + i];
        P.x[nxt][d * n + i] = xv;
        P.v[nxt][d * n + i] = vv;
        P.w[nxt][d * n + i] = wv;
        if (last) {
          P.out_v[d * n + i] = vv;
          P.out_w[d * n + i] = wv;
          P.out_F[d * n + i] = 0.0;
          P.out_M[d * n + i] = 0.0;
        }
      }
      P.act[nxt][i] = 0;
      for (int k = 0; k < 3; k++) RDo[3 * (size_t)i + k] = RD[3 * (size_t)i + k];
    } else {
      // every independent load first: the FP64 state and the owner sums do not depend on
      // the reactions, so their latencies overlap
      double xs[3], vs[3], ws[3];
      float us[6];
      for (int d = 0; d < 3; d++) {
        xs[d] = X[d * n + i];
        vs[d] = V[d * n + i];
        ws[d] = W[d * n + i];
        us[d] = P.upart[(size_t)d * n + i];
        us[3 + d] = P.upart[(size_t)(3 + d) * n + i];
      }
      const float Rif = P.rad[C->sbuf][i];
      // reactions pushed by the owners of the leading slots, in partner-id order
      const int ilo = P.inner_lo[i];
      float Ff[3] = {0.f, 0.f, 0.f}, Mf[3] = {0.f, 0.f, 0.f};
#pragma unroll 4
      for (int s = 0; s < ilo; s++) {
        const float4* r = P.rec + 2 * ((size_t)s * n + i);
        const float4 a = r[0], b = r[1];
        Ff[0] += a.x;
        Ff[1] += a.y;
        Ff[2] += a.z;
        Mf[0] += a.w;
        Mf[1] += b.x;
        Mf[2] += b.y;
      }
      for (int d = 0; d < 3; d++) {
        Ff[d] += us[d];
        Mf[d] += us[3 + d];
      }

      // ---------------- velocity Verlet in FP64 with FP32 accelerations (Eqs. main1, main2),
      // or explicit Euler (Eq. integ_EE: x^{n+1} = x^n + v^n dt, v^{n+1} = v^n + a^n dt)
      const float mif = P.f_density * (4.0f / 3.0f) * 3.14159265358979f * Rif * Rif * Rif;
      const float inv_m = 1.0f / mif;
      const float inv_I = 1.0f / (0.4f * mif * Rif * Rif);
      double xn[3], vn[3], wn[3];
      for (int d = 0; d < 3; d++) {
        const double xi = xs[d], vi = vs[d], wi = ws[d];
        const double a = f2d_int(Ff[d] * inv_m + P.f_g[d]);
        const double al = f2d_int(Mf[d] * inv_I);
        const bool euler = kExt && P.integrator == 1;
        if (init && !euler) {
          vn[d] = fma(a, P.half_dt, vi);
          wn[d] = fma(al, P.half_dt, wi);
        } else {
          vn[d] = fma(a, P.dt, vi);
          wn[d] = fma(al, P.dt, wi);
        }
        if (last) {
          P.out_v[d * n + i] = (init || euler) ? vi : fma(a, P.half_dt, vi);
          P.out_w[d * n + i] = (init || euler) ? wi : fma(al, P.half_dt, wi);
          P.out_F[d * n + i] = f2d_int(Ff[d]);
          P.out_M[d * n + i] = f2d_int(Mf[d]);
        }
        xn[d] = fma(euler ? vi : vn[d], P.dt, xi);
        P.x[nxt][d * n + i] = xn[d];
        P.v[nxt][d * n + i] = vn[d];
        P.w[nxt][d * n + i] = wn[d];
      }
      const bool alive = !below_sink(xn[2], P.z_sink_key);
      P.act[nxt][i] = alive ? 1 : 0;
      float hn[3], ln[3];
      for (int d = 0; d < 3; d++) split_df(xn[d], hn[d], ln[d]);
      write_render(RDo + 3 * (size_t)i, hn, ln, vn, wn, alive);
      if (!(finite_d(xn[0]) && finite_d(xn[1]) && finite_d(xn[2]) && finite_d(vn[0]) && finite_d(vn[1]) &&
            finite_d(vn[2])))
        st.status |= kStNonfinite;
      if (alive) {
        st.active++;
        const float dm = moved_since_inner(P.xin, n, i, hn, ln);
        if (dm * dm > P.f_inner_lim2) P.ctl->need_inner = 1;
        if (P.rebuild_every <= 0 && dm + P.xin[3 * (size_t)n + i] > P.f_disp_lim * (1.0f - 1e-5f)) {
          const float* xs = reinterpret_cast<const float*>(P.xref);
          float e2 = 0.f;
          for (int d = 0; d < 3; d++) {
            float s1, t1;
            df_diff(xs[d * n + i], xs[(3 + d) * n + i], hn[d], ln[d], s1, t1);
            const float u = s1 + t1;
            e2 += u * u;
          }
          if (e2 > P.f_disp_lim2) P.ctl->need_rebuild = 1;
        }
      }
    }
  }
  (void)hc;
  end_step(st, P.ctl, last, true);
}

void launch_step_mixed(const Params& P, cudaStream_t s) {
  const int T = P.step_block > 0 ? P.step_block : step_block(P.n, P.sm_count);
  const int blocks = (P.n + T - 1) / T;
  // the paper's other options (linear model, viscous rolling, explicit Euler, translating
  // walls) run in their own instantiation, so the default one keeps its registers
  const bool ext = P.contact_model != 0 || P.rolling == 2 || P.integrator != 0 || P.any_translating;
  if (P.pair_once) {
    if (P.n_inst > 1) {
      if (ext)
        k_pair_mixed<true, true><<<blocks, T, 0, s>>>(P);
      else
        k_pair_mixed<true, false><<<blocks, T, 0, s>>>(P);
    } else {
      if (ext)
        k_pair_mixed<false, true><<<blocks, T, 0, s>>>(P);
      else
        k_pair_mixed<false, false><<<blocks, T, 0, s>>>(P);
    }
    const int bi = (P.n + kIntBlock - 1) / kIntBlock;
    if (ext)
      k_int_mixed<true><<<bi, kIntBlock, 0, s>>>(P);
    else
      k_int_mixed<false><<<bi, kIntBlock, 0, s>>>(P);
    return;
  }
  if (P.n_inst > 1) {
    if (ext)
      k_step_mixed<true, true><<<blocks, T, 0, s>>>(P);
    else
      k_step_mixed<true, false><<<blocks, T, 0, s>>>(P);
  } else {
    if (ext)
      k_step_mixed<false, true><<<blocks, T, 0, s>>>(P);
    else
      k_step_mixed<false, false><<<blocks, T, 0, s>>>(P);
  }
}

}  // namespace demgb
