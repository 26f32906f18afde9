// dem_step_mixed.cu -- mixed-precision step kernel: FP32 contact law, FP64 positions,
// velocities, integration and tangential-overlap accumulation.
//
// One thread owns one particle of the cell-sorted order and walks its fine-search list.
// FP64 instructions issue at 1/72 of the FP32 rate on this part, so the kernel keeps them
// to the integration (9 FMAs per particle) and the tangential-overlap accumulation
// (3 adds per contact):
//   - relative positions and velocities come from integer splits of the FP64 values into
//     FP32 pairs (hi + lo) and exact two-sum differences, so nearly co-located or
//     co-moving spheres keep their relative values to ~1e-7;
//   - the normal overlap is (S^2 - r^2) / (S + r) with S^2 - r^2 formed exactly as a
//     double-float (no cancellation at small overlaps);
//   - FP32<->FP64 conversions use integer operations; uniform constants arrive in FP32;
//     the rebuild trigger, the z_sink test and the wall time windows use no FP64 work.
#include "dem_step_common.cuh"

namespace demgb {

__global__ void __launch_bounds__(kStepBlock, 7) k_step_mixed(Params P) {
  const Control* C = P.ctl;
  const int cur = C->cur, nxt = cur ^ 1, sb = C->sbuf, hc = C->hc;
  const bool init = C->init != 0, last = C->last != 0;
  const unsigned wall_on = C->wall_on;
  const int n = P.n, nact = C->n_act_sorted;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  StepStats st = {0u, 0u, 0u, 0.0f, 0u};
  const double* X = P.x[cur];
  const double* V = P.v[cur];
  const double* W = P.w[cur];
  const uint8_t* A = P.act[cur];
  const float* RAD = P.rad[sb];

  if (last && i >= nact && i < n) {
    for (int d = 0; d < 3; d++) {   // out of the system: frozen in both buffers
      P.out_v[d * n + i] = V[d * n + i];
      P.out_w[d * n + i] = W[d * n + i];
      P.out_F[d * n + i] = 0.0;
      P.out_M[d * n + i] = 0.0;
    }
  }
  if (i < nact) {
    double xi[3], vi[3], wi[3];
    for (int d = 0; d < 3; d++) {
      xi[d] = X[d * n + i];
      vi[d] = V[d * n + i];
      wi[d] = W[d * n + i];
    }
    if (!A[i]) {
      for (int d = 0; d < 3; d++) {
        P.x[nxt][d * n + i] = xi[d];
        P.v[nxt][d * n + i] = vi[d];
        P.w[nxt][d * n + i] = wi[d];
        if (last) {
          P.out_v[d * n + i] = vi[d];
          P.out_w[d * n + i] = wi[d];
          P.out_F[d * n + i] = 0.0;
          P.out_M[d * n + i] = 0.0;
        }
      }
      P.act[nxt][i] = 0;
      P.mask[hc ^ 1][i] = 0ull;
      P.shadow[nxt][i] = P.shadow[cur][i];
    } else {
      const unsigned long long mold = P.mask[hc][i];
      const double* Hold = P.hist[hc] + (size_t)i * kHistStride * 3;
      double* Hnew = P.hist[hc ^ 1] + (size_t)i * kHistStride * 3;
      const int* nb = P.nbr + (size_t)i * kMaxNbr;
      const int cnt = P.nbr_cnt[i];
      const float Rif = RAD[i];
      const float mif = P.f_density * (4.0f / 3.0f) * 3.14159265358979f * Rif * Rif * Rif;
      float hx[3], lx[3], vh[3], vl[3], wh[3], wl[3];
      for (int d = 0; d < 3; d++) {
        split_df(xi[d], hx[d], lx[d]);
        split_df(vi[d], vh[d], vl[d]);
        split_df(wi[d], wh[d], wl[d]);
      }
      const float wif[3] = {wh[0] + wl[0], wh[1] + wl[1], wh[2] + wl[2]};
      const float dtf = P.f_dt;
      float Ff[3] = {0.f, 0.f, 0.f}, Mf[3] = {0.f, 0.f, 0.f};
      unsigned long long mnew = 0ull;
      int rank = 0;

      // ---------------- particle-particle contacts
      // (a) Prefilter on the FP32 hi parts, 8 list entries at a time: two 16-byte loads of
      //     indices, then 8 independent 16-byte shadow loads.  hi truncates x to 24
      //     significant bits: |x - hi| < 2^-23 |x|, so a coordinate difference of two hi
      //     parts (partners within r_c) is off by less than 2^-23 (2 |x_i| + 2 r_c),
      //     rounding included; the test is widened by sqrt(3) times that bound, so it
      //     cannot drop a contact.
      const float4* SH = P.shadow[cur];
      const float amax = fmaxf(fmaxf(fabsf(hx[0]), fabsf(hx[1])), fabsf(hx[2]));
      const float slack = 1.7320508f * 1.1920929e-7f * (2.0f * amax + 2.0f * P.f_rc) + 1e-30f;
      const int4* nb4 = reinterpret_cast<const int4*>(nb);
      unsigned long long cand = 0ull;
      for (int k0 = 0; k0 < cnt; k0 += 8) {
        const int4 ja = nb4[k0 >> 2], jb = nb4[(k0 >> 2) + 1];   // row has 56 slots: in bounds
        const int js[8] = {ja.x, ja.y, ja.z, ja.w, jb.x, jb.y, jb.z, jb.w};
        float4 sh[8];
#pragma unroll
        for (int u = 0; u < 8; u++) sh[u] = (k0 + u < cnt) ? SH[js[u]] : make_float4(1e30f, 1e30f, 1e30f, 0.f);
#pragma unroll
        for (int u = 0; u < 8; u++) {
          const float ex = sh[u].x - hx[0], ey = sh[u].y - hx[1], ez = sh[u].z - hx[2];
          const float reach = (Rif + sh[u].w + slack) * 1.000001f;
          if (k0 + u < cnt && ex * ex + ey * ey + ez * ez < reach * reach) cand |= 1ull << (k0 + u);
        }
      }
      // (b) candidates in list order; every load of a candidate is issued before any branch
      while (cand) {
        const int k = __ffsll((long long)cand) - 1;
        cand &= cand - 1ull;
        const int j = nb[k];
        const bool had = (mold >> k) & 1ull;
        const int ro = __popcll(mold & ((1ull << k) - 1ull));
        const uint8_t aj = A[j];
        const float Rjf = RAD[j];
        double xj[3], vj[3], wjd[3];
        for (int d = 0; d < 3; d++) {
          xj[d] = X[(size_t)d * n + j];
          vj[d] = V[(size_t)d * n + j];
          wjd[d] = W[(size_t)d * n + j];
        }
        double H[3] = {0.0, 0.0, 0.0};
        if (had) {
          H[0] = Hold[ro * 3];
          H[1] = Hold[ro * 3 + 1];
          H[2] = Hold[ro * 3 + 2];
        }
        if (!aj) continue;
        float s[3], t[3], dxf[3];
        for (int d = 0; d < 3; d++) {
          float hj, lj;
          split_df(xj[d], hj, lj);
          df_diff(hx[d], lx[d], hj, lj, s[d], t[d]);
          dxf[d] = s[d] + t[d];
        }
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
        // v_i - v_j and w_i - w_j as exact double-float differences
        float dv[3], dw[3], wj[3];
        for (int d = 0; d < 3; d++) {
          float h, l, s1, t1;
          split_df(vj[d], h, l);
          df_diff(h, l, vh[d], vl[d], s1, t1);
          dv[d] = s1 + t1;
          split_df(wjd[d], h, l);
          wj[d] = h + l;
          df_diff(h, l, wh[d], wl[d], s1, t1);
          dw[d] = s1 + t1;
        }
        const float rw[3] = {Rif * wif[0] + Rjf * wj[0], Rif * wif[1] + Rjf * wj[1], Rif * wif[2] + Rjf * wj[2]};
        const float vij[3] = {dv[0] + (rw[1] * nrm[2] - rw[2] * nrm[1]), dv[1] + (rw[2] * nrm[0] - rw[0] * nrm[2]),
                              dv[2] + (rw[0] * nrm[1] - rw[1] * nrm[0])};
        const float Re = Rif * Rjf / S;
        const float mj = P.f_density * (4.0f / 3.0f) * 3.14159265358979f * Rjf * Rjf * Rjf;
        const float me = mif * mj / (mif + mj);
        law_f(nrm, dn, vij, dw, Re, me, P.f_Ye_pp, P.f_Ge_pp, P.f_ceta_pp, P.f_mu_pp, P.f_mur_pp, P.rolling, dtf, H,
              !init, Rif, Ff, Mf);
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
      }

      // ---------------- particle-wall contacts (FP32 prefilter, FP64 geometry)
      const float xf[3] = {hx[0] + lx[0], hx[1] + lx[1], hx[2] + lx[2]};
      for (int k = 0; k < P.n_walls; k++) {
        if (!((wall_on >> k) & 1u)) continue;
        if (!wall_maybe_f(P.walls[k].kind, P.wf[k], xf, Rif, P.wall_margin)) continue;
        const WallDev& Wl = P.walls[k];
        double nrmd[3], dnd, ps[3];
        if (!wall_geom_d(Wl, xi, (double)Rif, nrmd, &dnd, ps)) continue;
        const double arm[3] = {ps[0] - Wl.c[0], ps[1] - Wl.c[1], ps[2] - Wl.c[2]};
        double Vw[3];
        cross3d(Wl.Om, arm, Vw);
        for (int d = 0; d < 3; d++) Vw[d] += Wl.V[d];
        const int bit = kMaxNbr + k;
        double H[3] = {0.0, 0.0, 0.0};
        if ((mold >> bit) & 1ull) {
          const int ro = __popcll(mold & ((1ull << bit) - 1ull));
          H[0] = Hold[ro * 3];
          H[1] = Hold[ro * 3 + 1];
          H[2] = Hold[ro * 3 + 2];
        }
        const float nf[3] = {(float)nrmd[0], (float)nrmd[1], (float)nrmd[2]};
        const float dnf = (float)dnd;
        float dv[3], dw[3];
        for (int d = 0; d < 3; d++) {
          float h, l, s1, t1;
          split_df(Vw[d], h, l);
          df_diff(h, l, vh[d], vl[d], s1, t1);       // v_i - V_wall(p*)
          dv[d] = s1 + t1;
          split_df(Wl.Om[d], h, l);
          df_diff(h, l, wh[d], wl[d], s1, t1);       // w_i - Omega
          dw[d] = s1 + t1;
        }
        const float rw[3] = {Rif * wif[0], Rif * wif[1], Rif * wif[2]};
        const float vij[3] = {dv[0] + (rw[1] * nf[2] - rw[2] * nf[1]), dv[1] + (rw[2] * nf[0] - rw[0] * nf[2]),
                              dv[2] + (rw[0] * nf[1] - rw[1] * nf[0])};
        law_f(nf, dnf, vij, dw, Rif, mif, P.f_Ye_pw, P.f_Ge_pw, P.f_ceta_pw, P.f_mu_pw, P.f_mur_pw, P.rolling, dtf, H,
              !init, Rif, Ff, Mf);
        st.max_ovl = fmaxf(st.max_ovl, dnf / Rif);
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

      // ---------------- velocity Verlet in FP64 with FP32 accelerations (Eqs. main1, main2)
      const float inv_m = 1.0f / mif;
      const float inv_I = 1.0f / (0.4f * mif * Rif * Rif);
      double xn[3], vn[3], wn[3];
      for (int d = 0; d < 3; d++) {
        const double a = f2d_int(Ff[d] * inv_m + P.f_g[d]);
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
          P.out_F[d * n + i] = f2d_int(Ff[d]);
          P.out_M[d * n + i] = f2d_int(Mf[d]);
        }
        xn[d] = fma(vn[d], P.dt, xi[d]);
        P.x[nxt][d * n + i] = xn[d];
        P.v[nxt][d * n + i] = vn[d];
        P.w[nxt][d * n + i] = wn[d];
      }
      P.shadow[nxt][i] = make_float4(hi_df(xn[0]), hi_df(xn[1]), hi_df(xn[2]), Rif);
      const bool alive = !below_sink(xn[2], P.z_sink_key);
      P.act[nxt][i] = alive ? 1 : 0;
      if (!(finite_d(xn[0]) && finite_d(xn[1]) && finite_d(xn[2]) && finite_d(vn[0]) && finite_d(vn[1]) &&
            finite_d(vn[2])))
        st.status |= kStNonfinite;
      if (alive) {
        st.active++;
        // dynamic search trigger |x^{n+1} - x_ref|^2 > (skin/2)^2 without FP64 arithmetic
        float d2 = 0.f;
        for (int d = 0; d < 3; d++) {
          float ah, al, bh, bl, s1, t1;
          split_df(P.xref[d * n + i], ah, al);
          split_df(xn[d], bh, bl);
          df_diff(ah, al, bh, bl, s1, t1);
          const float u = s1 + t1;
          d2 += u * u;
        }
        if (P.rebuild_every <= 0 && d2 > P.f_disp_lim2) P.ctl->need_rebuild = 1;
      }
    }
  }
  if (P.max_overlap_ratio > 0.0 && st.max_ovl > (float)P.max_overlap_ratio) st.status |= kStOverlap;
  block_flush(st, P.ctl);
  finish_step(P.ctl);
}

void launch_step_mixed(const Params& P, cudaStream_t s) {
  const int blocks = (P.n + kStepBlock - 1) / kStepBlock;
  k_step_mixed<<<blocks, kStepBlock, 0, s>>>(P);
}

}  // namespace demgb
