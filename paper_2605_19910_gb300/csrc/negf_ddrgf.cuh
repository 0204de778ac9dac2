// DDRGF (Sec. 3, Alg. 2) schedule of one energy range (one TU: included by
// negf_capi.cu only), with the plan's DDRGF workspace layout.
#pragma once

#include "negf_sweep.cuh"

namespace {

// ---------------------------------------------------------------------------
// Layout.  The chain is cut into n_domains (D2, D1) pairs (Fig.
// parallel_RGF_domains): D2_j = [dom_f[j], dom_l[j]] followed by its
// separator D1_j of w layers.  F_j / L_j are the first / last w layers of
// D2_j, P_j the separator's layers as one super-block.
//
// Step 1 works on each closed sub-domain cut into w-layer groups (a block
// tridiagonal chain of super-blocks, Sec. 2.3 block fusing): anchored at the
// first layer for the right-connected sweep (the last group may be shorter)
// and at the last layer for the left-connected sweep (the first group may be
// shorter).  Eliminating whole w-layer groups pivots across the group, which
// keeps the closed sub-domains' corners accurate near their resonances.
// ---------------------------------------------------------------------------

// Fills the DDRGF part of the plan (domain layout already in dom_f / dom_l,
// interface levels in lvl).  Returns 0, -1 for interface levels that cut a
// chain into pairs of fewer than two nodes, 1 if a super-block exceeds the
// inversion kernel's limit.
inline int dd_layout(negf_plan_s* p, int max_block) {
  const int N = p->N, w = p->w, nd = p->n_domains;
  p->dom_of.assign(N, -1); p->sep_of.assign(N, -1); p->off_in.assign(N, 0);
  p->Fsz.assign(nd, 0); p->Lsz.assign(nd, 0); p->Psz.assign(nd, 0);
  for (int j = 0; j < nd; ++j) {
    for (int a = p->dom_f[j]; a <= p->dom_l[j]; ++a) p->dom_of[a] = j;
    for (int r = 0; r < w; ++r) {
      p->off_in[p->dom_f[j] + r] = p->Fsz[j];
      p->Fsz[j] += p->b[p->dom_f[j] + r];
      p->Lsz[j] += p->b[p->dom_l[j] - w + 1 + r];
      const int sl = p->dom_l[j] + 1 + r;
      p->sep_of[sl] = j;
      p->off_in[sl] = p->Psz[j];
      p->Psz[j] += p->b[sl];
    }
    p->Pmax = std::max(p->Pmax, p->Psz[j]);
    p->FLmax = std::max(p->FLmax, std::max(p->Fsz[j], p->Lsz[j]));
  }
  p->dd_e = 0;
  p->hf_e = 0;
  auto reg = [&](int64_t size) { negf_plan_s::Reg r{p->dd_e, size}; p->dd_e += size; return r; };
  auto hreg = [&](int64_t size) { const int64_t o = p->hf_e; p->hf_e += size; return o; };
  p->grR.assign(nd, DDGroups());
  p->grL.assign(nd, DDGroups());
  p->Bmax = 0;
  for (int j = 0; j < nd; ++j) {
    const int f = p->dom_f[j], l = p->dom_l[j];
    for (int side = 0; side < 2; ++side) {
      DDGroups& g = side == 0 ? p->grR[j] : p->grL[j];
      std::vector<std::pair<int, int>> ranges;   // [lo, hi] layers of each group, in chain order
      if (side == 0)
        for (int lo = f; lo <= l; lo += w) ranges.push_back({lo, std::min(l, lo + w - 1)});
      else {
        for (int hi = l; hi >= f; hi -= w) ranges.push_back({std::max(f, hi - w + 1), hi});
        std::reverse(ranges.begin(), ranges.end());
      }
      for (auto& rg : ranges) {
        int sz = 0;
        for (int a = rg.first; a <= rg.second; ++a) sz += p->b[a];
        g.first.push_back(rg.first);
        g.nl.push_back(rg.second - rg.first + 1);
        g.sz.push_back(sz);
        p->Bmax = std::max(p->Bmax, sz);
      }
      const int K = (int)g.sz.size();
      for (int I = 0; I < K; ++I) {
        g.hd.push_back(hreg(sq(g.sz[I])));
        g.hu.push_back(I + 1 < K ? hreg((int64_t)g.sz[I] * g.sz[I + 1]) : -1);
        g.hl.push_back(I + 1 < K ? hreg((int64_t)g.sz[I + 1] * g.sz[I]) : -1);
        if (side == 0) {
          g.t.push_back(reg(sq(g.sz[I])));
          g.x.push_back(I > 0 ? reg((int64_t)g.sz[I] * g.sz[I - 1]) : negf_plan_s::Reg{});
          g.y.push_back(I > 0 ? reg((int64_t)g.sz[I - 1] * g.sz[I]) : negf_plan_s::Reg{});
        }
      }
    }
  }
  if (p->Bmax > max_block || p->Pmax > max_block || p->FLmax > max_block) return 1;
  const int64_t B2 = sq(p->Bmax);
  p->r_xll.resize(nd); p->r_xfl.resize(nd); p->r_xlf.resize(nd);
  p->r_lsS.resize(nd); p->r_lsG.resize(nd); p->r_lsY.resize(nd); p->r_row.resize(nd); p->r_col.resize(nd);
  p->r_wr.resize(nd); p->r_vr.resize(nd); p->r_sr.resize(nd); p->r_wl.resize(nd); p->r_vl.resize(nd);
  p->r_sl.resize(nd); p->r_tmp.resize(nd);
  for (int j = 0; j < nd; ++j) {
    const int F = p->Fsz[j], L = p->Lsz[j], P = p->Psz[j], P0 = j > 0 ? p->Psz[j - 1] : 0;
    p->r_xll[j] = reg(sq(L));
    p->r_xfl[j] = reg((int64_t)F * L);
    p->r_xlf[j] = reg((int64_t)L * F);
    p->r_lsS[j] = reg(B2);
    p->r_lsG[j] = reg(B2);
    p->r_lsY[j] = reg(B2);
    p->r_row[j] = reg(2 * (int64_t)F * p->Bmax);
    p->r_col[j] = reg(2 * (int64_t)p->Bmax * F);
    p->r_wr[j] = reg((int64_t)L * P);
    p->r_vr[j] = reg((int64_t)P * L);
    p->r_sr[j] = reg(sq(L));
    p->r_wl[j] = reg((int64_t)F * P0);
    p->r_vl[j] = reg((int64_t)P0 * F);
    p->r_sl[j] = reg(sq(F));
    p->r_tmp[j] = reg((int64_t)p->Pmax * p->FLmax);
  }
  p->r_A.resize(nd); p->r_cL.resize(nd); p->r_cR.resize(nd); p->r_base.resize(nd); p->r_LL.resize(nd);
  p->r_RR.resize(nd); p->r_gLs.resize(nd); p->r_gRin.resize(nd); p->r_gRs.resize(nd);
  p->r_Gpp.resize(nd); p->r_Tu.resize(nd); p->r_Tl.resize(nd);
  for (int k = 0; k < nd; ++k) {
    const int64_t P2 = sq(p->Psz[k]), PP = k + 1 < nd ? (int64_t)p->Psz[k] * p->Psz[k + 1] : 0;
    p->r_A[k] = reg(P2); p->r_cL[k] = reg(P2); p->r_cR[k] = reg(P2); p->r_base[k] = reg(P2);
    p->r_LL[k] = reg(P2); p->r_RR[k] = reg(P2); p->r_gLs[k] = reg(P2);
    p->r_gRin[k] = reg(P2); p->r_gRs[k] = reg(P2); p->r_Gpp[k] = reg(P2);
    p->r_Tu[k] = reg(PP); p->r_Tl[k] = reg(PP);
  }
  // interface levels: chain 0 is the separators' chain (T_S); a level with a
  // pair count in lvl is cut into pairs and its separators form the next chain
  p->chains.assign(1, DDChain());
  {
    DDChain& c0 = p->chains[0];
    c0.n = nd;
    c0.sz = p->Psz;
    c0.D = p->r_base;
    c0.U.assign(p->r_Tu.begin(), p->r_Tu.end() - 1);
    c0.L.assign(p->r_Tl.begin(), p->r_Tl.end() - 1);
    c0.LL = p->r_LL;
    c0.RR = p->r_RR;
  }
  const int64_t PM2 = sq(p->Pmax);
  for (size_t k = 0; k < p->chains.size(); ++k) {
    const int n = p->chains[k].n;
    std::vector<int> sz = p->chains[k].sz;
    std::vector<negf_plan_s::Reg> t(n), X(n), Y(n), tmp(n);
    for (int i = 0; i < n; ++i) {
      t[i] = reg(sq(sz[i]));
      tmp[i] = reg(PM2);
      if (i > 0) { X[i] = reg((int64_t)sz[i] * sz[i - 1]); Y[i] = reg((int64_t)sz[i - 1] * sz[i]); }
    }
    p->chains[k].t = t; p->chains[k].X = X; p->chains[k].Y = Y; p->chains[k].tmp = tmp;
    if (k >= p->lvl.size()) continue;              // the deepest level: sequential sweeps
    const int np = p->lvl[k];
    std::vector<int> f(np), l(np), nsz(np);
    for (int J = 0; J < np; ++J) {
      const int lo = (int)((int64_t)J * n / np), hi = (int)((int64_t)(J + 1) * n / np);   // pair = [lo, hi)
      if (hi - lo < 2) return -1;
      f[J] = lo; l[J] = hi - 2;
      nsz[J] = sz[hi - 1];
    }
    std::vector<negf_plan_s::Reg> row(np), col(np), xll(np), s1(np), s2(np), cL(n), cR(n);
    for (int J = 0; J < np; ++J) {
      row[J] = reg(2 * (int64_t)sz[f[J]] * p->Pmax);
      col[J] = reg(2 * (int64_t)p->Pmax * sz[f[J]]);
      xll[J] = reg(sq(sz[l[J]]));
      s1[J] = reg(PM2);
      s2[J] = reg(PM2);
      const int q = l[J] + 1;
      cL[q] = reg(sq(sz[q]));
      cR[q] = reg(sq(sz[q]));
    }
    DDChain h;
    h.n = np;
    h.sz = nsz;
    for (int q = 0; q < np; ++q) {
      h.D.push_back(reg(sq(nsz[q])));
      h.LL.push_back(reg(sq(nsz[q])));
      h.RR.push_back(reg(sq(nsz[q])));
      if (q + 1 < np) {
        h.U.push_back(reg((int64_t)nsz[q] * nsz[q + 1]));
        h.L.push_back(reg((int64_t)nsz[q + 1] * nsz[q]));
      }
    }
    DDChain& c = p->chains[k];
    c.np = np; c.f = f; c.l = l;
    c.row = row; c.col = col; c.xll = xll; c.s1 = s1; c.s2 = s2; c.cL = cL; c.cR = cR;
    c.child = (int)p->chains.size();
    p->chains.push_back(h);                        // may reallocate: no reference kept across
  }
  if ((int)p->chains.size() != (int)p->lvl.size() + 1) return -1;
  p->r_g1 = reg(2 * (int64_t)p->b[0] * p->Pmax);
  p->r_g1t = reg((int64_t)p->b[0] * p->Pmax);
  // energy-independent M super-blocks between F / L and the separators
  p->mfp_off.assign(nd, 0); p->mpf_off.assign(nd, 0); p->mlq_off.assign(nd, 0); p->mql_off.assign(nd, 0);
  for (int j = 0; j < nd; ++j) {
    const int Pp = j > 0 ? p->Psz[j - 1] : 0;
    p->mfp_off[j] = hreg((int64_t)p->Fsz[j] * Pp);
    p->mpf_off[j] = hreg((int64_t)Pp * p->Fsz[j]);
    p->mlq_off[j] = hreg((int64_t)p->Lsz[j] * p->Psz[j]);
    p->mql_off[j] = hreg((int64_t)p->Psz[j] * p->Lsz[j]);
  }
  return 0;
}

// ---------------------------------------------------------------------------
// DDRGF for one energy range:
//   step 1: per sub-domain (concurrently), the corner super-blocks X_FF,
//           X_FL, X_LF, X_LL of the closed sub-domain's inverse (fused
//           right- and left-connected sweeps, first super-row / column
//           chains);
//   steps 2-3: the interface system T_S = T11 - T12 X T21 (Eq.
//           Schur_complement_in_parallel_DDRGF; block tridiagonal over the
//           separators, Prop. 4), FP64: its left- and right-connected sweeps
//           and the separator diagonals of T_S^{-1}; every matrix that is
//           inverted is formed from its own parts;
//   step 4: the four parts of Eq. 2x2_explicit_inverse_parallel_DDRGF on the
//           band, evaluated as each sub-domain's RGF with the boundary
//           self-energies Sigma_left = M_{F,p} gL_p M_{p,F} and Sigma_right =
//           M_{L,q} gR_q M_{q,L} of the rest of the chain (gL_p / gR_q: the
//           interface's connected Green's functions at the neighbouring
//           separators without this sub-domain), plus the blocks between the
//           sub-domain and its separators.  Equal in exact arithmetic to the
//           stitching G_22 = X + X T21 T_S^{-1} T12 X, without adding the
//           closed sub-domain's inverse to a term that cancels it.
// ---------------------------------------------------------------------------
struct DD {
  negf_plan_s* p;
  Sweep& s;
  int w, nd, C;
  int64_t sG;

  DD(negf_plan_s* pp, Sweep& ss) : p(pp), s(ss), w(pp->w), nd(pp->n_domains), C(ss.ne), sG(pp->band_elems) {}

  int b(int i) const { return p->b[i]; }
  double2* R(const negf_plan_s::Reg& r) const { return p->DDW + r.off * p->chunk + (int64_t)s.wofs * r.sz; }
  const double2* HF(int64_t off) const { return p->Hf + off; }
  int offL(int c) const {          // offset of layer c inside L of its domain
    const int j = p->dom_of[c];
    int o = 0;
    for (int k = p->dom_l[j] - w + 1; k < c; ++k) o += b(k);
    return o;
  }
  int offF(int c) const { return p->off_in[c]; }   // offset of layer c inside F of its domain

  // C (+)= alpha A B over the range's energies (per-energy strides, 0 =
  // shared operand).  kind: 0 FP64, 1 plan precision, 2 step-1 precision
  // (FP64, or 56-bit tensor-core products on mixed plans).
  cudaError_t mm(int kind, int m, int n, int k, const double2* A, int64_t sA, int lda, const double2* B, int64_t sB,
                 int ldb, double2* Cm, int64_t sC, int ldc, double alpha, bool acc = false,
                 const double2* C1 = nullptr, int64_t sC1 = 0, int ldc1 = 0, double beta1 = 1.0,
                 const double2* dshift = nullptr) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    ZGemm g;
    g.m = m; g.n = n; g.k = k;
    g.A = A; g.sA = sA; g.lda = lda;
    g.B = B; g.sB = sB; g.ldb = ldb;
    g.C = Cm; g.sC = sC; g.ldc = ldc;
    g.alpha = {alpha, 0.0};
    if (C1) { g.C1 = C1; g.sC1 = sC1; g.ldc1 = ldc1; g.beta1 = {beta1, 0.0}; }
    else if (acc) { g.C1 = Cm; g.sC1 = sC; g.ldc1 = ldc; g.beta1 = {1.0, 0.0}; }
    if (dshift) { g.dshift = dshift; g.sD = 1; g.gamma = {1.0, 0.0}; }
    g.batch = C;
    if (kind == 1) return s.gemm(g);
    if (kind == 2 && p->precision == NEGF_MIXED) { g.bits = 56; return s.gemm(g); }
    return s.gemm64(g);
  }
  cudaError_t cp(const double2* src, int64_t sSrc, int ldSrc, double2* dst, int64_t sDst, int ldDst, int rows,
                 int cols, double scale, int acc, int batch) {
    return s.misc([&] { return negf::copy2d(src, sSrc, ldSrc, dst, sDst, ldDst, rows, cols, scale, acc, batch, s.st); });
  }
  cudaError_t zero(double2* dst, int64_t sDst, int ld, int rows, int cols, int batch) {
    return s.misc([&] { return negf::set_eye(dst, sDst, ld, rows, cols, 0, 0, 0, batch, s.st); });
  }
  cudaError_t comb(const negf_plan_s::Reg& out, int64_t n, const negf_plan_s::Reg* r0, double c0,
                   const negf_plan_s::Reg* r1, double c1, const negf_plan_s::Reg* r2, double c2,
                   const negf_plan_s::Reg* r3, double c3) {
    auto ptr = [&](const negf_plan_s::Reg* r) -> const double2* { return r ? R(*r) : nullptr; };
    auto str = [&](const negf_plan_s::Reg* r) -> int64_t { return r ? r->sz : 0; };
    return s.misc([&] {
      return negf::lincomb(R(out), out.sz, n, C, ptr(r0), str(r0), c0, ptr(r1), str(r1), c1, ptr(r2), str(r2), c2,
                           ptr(r3), str(r3), c3, s.st);
    });
  }
  // In-place inversion of a separator super-block (info: the separator's first layer).
  cudaError_t inv_reg(const negf_plan_s::Reg& r, int k) {
    return s.inv(R(r), r.sz, R(r), r.sz, p->Psz[k], C, p->dom_l[k] + 2);
  }

  // Energy-independent blocks: the fused H super-blocks of step 1 and the M
  // super-blocks between F / L and the separators.
  cudaError_t assemble_static() {
    auto fused = [&](int64_t off, int r0, int nr, int c0, int nc, int rows, int cols) -> cudaError_t {
      double2* dst = p->Hf + off;
      NEGF_TRY(zero(dst, 0, cols, rows, cols, 1));
      int ro = 0;
      for (int a = r0; a < r0 + nr; ++a) {
        int co = 0;
        for (int c = c0; c < c0 + nc; ++c) {
          if (std::abs(a - c) <= w) NEGF_TRY(cp(s.Hblk(a, c), 0, b(c), dst + (int64_t)ro * cols + co, 0, cols, b(a), b(c),
                                                1.0, 0, 1));
          co += b(c);
        }
        ro += b(a);
      }
      return cudaSuccess;
    };
    for (int j = 0; j < nd; ++j)
      for (int side = 0; side < 2; ++side) {
        const DDGroups& g = side == 0 ? p->grR[j] : p->grL[j];
        const int K = (int)g.sz.size();
        for (int I = 0; I < K; ++I) {
          NEGF_TRY(fused(g.hd[I], g.first[I], g.nl[I], g.first[I], g.nl[I], g.sz[I], g.sz[I]));
          if (I + 1 < K) {
            NEGF_TRY(fused(g.hu[I], g.first[I], g.nl[I], g.first[I + 1], g.nl[I + 1], g.sz[I], g.sz[I + 1]));
            NEGF_TRY(fused(g.hl[I], g.first[I + 1], g.nl[I + 1], g.first[I], g.nl[I], g.sz[I + 1], g.sz[I]));
          }
        }
      }
    for (int j = 0; j < nd; ++j) {
      const int f = p->dom_f[j], l = p->dom_l[j], F = p->Fsz[j], L = p->Lsz[j], P = p->Psz[j];
      const int P0 = j > 0 ? p->Psz[j - 1] : 0;
      double2* MFp = p->Hf + p->mfp_off[j];
      double2* MpF = p->Hf + p->mpf_off[j];
      double2* MLq = p->Hf + p->mlq_off[j];
      double2* MqL = p->Hf + p->mql_off[j];
      NEGF_TRY(zero(MLq, 0, P, L, P, 1));
      NEGF_TRY(zero(MqL, 0, L, P, L, 1));
      if (P0) {
        NEGF_TRY(zero(MFp, 0, P0, F, P0, 1));
        NEGF_TRY(zero(MpF, 0, F, P0, F, 1));
      }
      for (int r = l - w + 1; r <= l; ++r)
        for (int sl = l + 1; sl <= l + w; ++sl) {
          if (sl - r > w) continue;
          NEGF_TRY(cp(s.Hblk(r, sl), 0, b(sl), MLq + (int64_t)offL(r) * P + p->off_in[sl], 0, P, b(r), b(sl), -1.0, 0, 1));
          NEGF_TRY(cp(s.Hblk(sl, r), 0, b(r), MqL + (int64_t)p->off_in[sl] * L + offL(r), 0, L, b(sl), b(r), -1.0, 0, 1));
        }
      if (P0)
        for (int r = f; r < f + w; ++r)
          for (int sl = f - w; sl < f; ++sl) {
            if (r - sl > w) continue;
            NEGF_TRY(cp(s.Hblk(r, sl), 0, b(sl), MFp + (int64_t)offF(r) * P0 + p->off_in[sl], 0, P0, b(r), b(sl), -1.0, 0, 1));
            NEGF_TRY(cp(s.Hblk(sl, r), 0, b(r), MpF + (int64_t)p->off_in[sl] * F + offF(r), 0, F, b(sl), b(r), -1.0, 0, 1));
          }
    }
    return cudaSuccess;
  }

  // S_I = E I - H_II (fused), minus Sigma_L on layer 0 when the group holds it.
  cudaError_t diag_group(const DDGroups& g, int I, double2* S, int64_t sS) {
    const int B = g.sz[I];
    NEGF_TRY(mm(0, B, B, 0, S, sS, B, S, sS, B, S, sS, B, 1.0, false, HF(g.hd[I]), 0, B, -1.0, s.E + s.e0));
    if (g.first[I] == 0 && s.sigL)
      NEGF_TRY(cp(s.sigmaL(), s.sig_stride, b(0), S, sS, B, b(0), b(0), -1.0, 1, C));
    return cudaSuccess;
  }

  // Step 1 for domain j.
  cudaError_t corners(int j) {
    const DDGroups& g = p->grR[j];
    const int K = (int)g.sz.size(), F = p->Fsz[j], L = p->Lsz[j];
    double2* S = R(p->r_lsS[j]);
    const int64_t sS = p->r_lsS[j].sz;
    // right-connected sweep of the closed sub-domain on groups anchored at f
    NEGF_TRY(diag_group(g, K - 1, S, sS));
    for (int I = K - 1; I >= 0; --I) {
      const int B = g.sz[I];
      NEGF_TRY(s.inv(S, sS, R(g.t[I]), g.t[I].sz, B, C, g.first[I] + 1));
      if (I == 0) break;
      const int Bp = g.sz[I - 1];
      // Y_I = M_{I-1,I} t_I = -H_u t_I ; X_I = t_I M_{I,I-1} = -t_I H_l
      NEGF_TRY(mm(2, Bp, B, B, HF(g.hu[I - 1]), 0, B, R(g.t[I]), g.t[I].sz, B, R(g.y[I]), g.y[I].sz, B, -1.0));
      NEGF_TRY(mm(2, B, Bp, B, R(g.t[I]), g.t[I].sz, B, HF(g.hl[I - 1]), 0, Bp, R(g.x[I]), g.x[I].sz, Bp, -1.0));
      // S_{I-1} = E I - H_{I-1,I-1} + Y_I H_l
      NEGF_TRY(mm(2, Bp, Bp, B, R(g.y[I]), g.y[I].sz, B, HF(g.hl[I - 1]), 0, Bp, S, sS, Bp, 1.0, false,
                  HF(g.hd[I - 1]), 0, Bp, -1.0, s.E + s.e0));
      if (g.first[I - 1] == 0 && s.sigL)
        NEGF_TRY(cp(s.sigmaL(), s.sig_stride, b(0), S, sS, Bp, b(0), b(0), -1.0, 1, C));
    }
    // X_FF = t_0; first super-row X_{F,J} = -X_{F,J-1} Y_J and first
    // super-column X_{J,F} = -X_J X_{J-1,F} (rings of two), the last w
    // layers' columns / rows into X_FL / X_LF
    const int rL = g.sz[K - 1];                 // elements of L in the last group
    const int rP = L - rL;                      // elements of L in group K-2 (shorter last group)
    const int64_t srow = p->r_row[j].sz, scol = p->r_col[j].sz;
    const int64_t slotR = (int64_t)F * p->Bmax, slotC = (int64_t)p->Bmax * F;
    auto rowp = [&](int J) -> double2* { return J == 0 ? R(g.t[0]) : R(p->r_row[j]) + (J & 1) * slotR; };
    auto colp = [&](int J) -> double2* { return J == 0 ? R(g.t[0]) : R(p->r_col[j]) + (J & 1) * slotC; };
    auto rows_s = [&](int J) -> int64_t { return J == 0 ? g.t[0].sz : srow; };
    auto cols_s = [&](int J) -> int64_t { return J == 0 ? g.t[0].sz : scol; };
    for (int J = 1; J < K; ++J) {
      const int B = g.sz[J], Bp = g.sz[J - 1];
      NEGF_TRY(mm(2, F, B, Bp, rowp(J - 1), rows_s(J - 1), Bp, R(g.y[J]), g.y[J].sz, B, rowp(J), rows_s(J), B, -1.0));
      NEGF_TRY(mm(2, B, F, Bp, R(g.x[J]), g.x[J].sz, Bp, colp(J - 1), cols_s(J - 1), F, colp(J), cols_s(J), F, -1.0));
    }
    double2* XFL = R(p->r_xfl[j]);
    double2* XLF = R(p->r_xlf[j]);
    NEGF_TRY(cp(rowp(K - 1), rows_s(K - 1), rL, XFL + rP, p->r_xfl[j].sz, L, F, rL, 1.0, 0, C));
    NEGF_TRY(cp(colp(K - 1), cols_s(K - 1), F, XLF + (int64_t)rP * F, p->r_xlf[j].sz, F, rL, F, 1.0, 0, C));
    if (rP > 0) {
      const int Bq = g.sz[K - 2];
      NEGF_TRY(cp(rowp(K - 2) + (Bq - rP), rows_s(K - 2), Bq, XFL, p->r_xfl[j].sz, L, F, rP, 1.0, 0, C));
      NEGF_TRY(cp(colp(K - 2) + (int64_t)(Bq - rP) * F, cols_s(K - 2), F, XLF, p->r_xlf[j].sz, F, rP, F, 1.0, 0, C));
    }
    // left-connected sweep on groups anchored at l: X_LL = the last group's inverse
    const DDGroups& h = p->grL[j];
    const int KL = (int)h.sz.size();
    double2* Gm = R(p->r_lsG[j]);
    double2* Ym = R(p->r_lsY[j]);
    const int64_t sB = p->r_lsG[j].sz;
    NEGF_TRY(diag_group(h, 0, S, sS));
    for (int I = 0; I < KL; ++I) {
      const int B = h.sz[I];
      if (I == KL - 1) return s.inv(S, sS, R(p->r_xll[j]), p->r_xll[j].sz, B, C, h.first[I] + 1);
      NEGF_TRY(s.inv(S, sS, Gm, sB, B, C, h.first[I] + 1));
      const int Bn = h.sz[I + 1];
      // Y = M_{I+1,I} g_I = -H_l g_I ; S_{I+1} = E I - H_{I+1,I+1} + Y H_u
      NEGF_TRY(mm(2, Bn, B, B, HF(h.hl[I]), 0, B, Gm, sB, B, Ym, sB, B, -1.0));
      NEGF_TRY(mm(2, Bn, Bn, B, Ym, sB, B, HF(h.hu[I]), 0, Bn, S, sS, Bn, 1.0, false, HF(h.hd[I + 1]), 0, Bn, -1.0,
                  s.E + s.e0));
      if (h.first[I + 1] == 0 && s.sigL)
        NEGF_TRY(cp(s.sigmaL(), s.sig_stride, b(0), S, sS, Bn, b(0), b(0), -1.0, 1, C));
    }
    return cudaSuccess;
  }

  // Steps 2-3 (FP64): T_S pieces per separator, the left- and right-connected
  // sweeps over the separators, and the separator diagonals of T_S^{-1}.
  cudaError_t interface() {
    const int N = p->N;
    for (int k = 0; k < nd; ++k) {
      const int P = p->Psz[k], s0 = p->dom_l[k] + 1, Lk = p->Lsz[k];
      double2* A = R(p->r_A[k]);
      const int64_t sP = p->r_A[k].sz;
      // A_k = E I - H_PP (- Sigma_R on the last layer)
      NEGF_TRY(zero(A, sP, P, P, P, C));
      for (int a = s0; a < s0 + w; ++a)
        for (int c = s0; c < s0 + w; ++c)
          NEGF_TRY(cp(s.Hblk(a, c), 0, b(c), A + (int64_t)p->off_in[a] * P + p->off_in[c], sP, P, b(a), b(c), -1.0, 0, C));
      NEGF_TRY(s.misc([&] { return negf::add_diag(A, sP, P, P, s.E + s.e0, 1, 1.0, C, s.st); }));
      if (s0 + w - 1 == N - 1 && s.sigR)
        NEGF_TRY(cp(s.sigmaR(), s.sig_stride, b(N - 1), A + (int64_t)p->off_in[N - 1] * P + p->off_in[N - 1], sP, P,
                    b(N - 1), b(N - 1), -1.0, 1, C));
      double2* T = R(p->r_tmp[k]);
      const int64_t sT = p->r_tmp[k].sz;
      const double2* MqL = HF(p->mql_off[k]);
      const double2* MLq = HF(p->mlq_off[k]);
      // cL_k = M_{P,L} X_LL M_{L,P} (sub-domain k, left of separator k)
      NEGF_TRY(mm(0, P, Lk, Lk, MqL, 0, Lk, R(p->r_xll[k]), p->r_xll[k].sz, Lk, T, sT, Lk, 1.0));
      NEGF_TRY(mm(0, P, P, Lk, T, sT, Lk, MLq, 0, P, R(p->r_cL[k]), sP, P, 1.0));
      if (k + 1 < nd) {
        const int j = k + 1, F = p->Fsz[j], L = p->Lsz[j], P1 = p->Psz[j];
        const double2* MpF = HF(p->mpf_off[j]);
        const double2* MFp = HF(p->mfp_off[j]);
        // cR_k = M_{P,F} X_FF M_{F,P} (sub-domain k + 1, right of separator k)
        NEGF_TRY(mm(0, P, F, F, MpF, 0, F, R(p->grR[j].t[0]), p->grR[j].t[0].sz, F, T, sT, F, 1.0));
        NEGF_TRY(mm(0, P, P, F, T, sT, F, MFp, 0, P, R(p->r_cR[k]), sP, P, 1.0));
        // T_S[k, k+1] = -M_{P_k,F} X_FL M_{L,P_{k+1}},  T_S[k+1, k] = -M_{P_{k+1},L} X_LF M_{F,P_k}
        NEGF_TRY(mm(0, P, L, F, MpF, 0, F, R(p->r_xfl[j]), p->r_xfl[j].sz, L, T, sT, L, 1.0));
        NEGF_TRY(mm(0, P, P1, L, T, sT, L, HF(p->mlq_off[j]), 0, P1, R(p->r_Tu[k]), p->r_Tu[k].sz, P1, -1.0));
        NEGF_TRY(mm(0, P1, F, L, HF(p->mql_off[j]), 0, L, R(p->r_xlf[j]), p->r_xlf[j].sz, F, T, sT, F, 1.0));
        NEGF_TRY(mm(0, P1, P, F, T, sT, F, MFp, 0, P, R(p->r_Tl[k]), p->r_Tl[k].sz, P, -1.0));
      }
      // base_k = A_k - cL_k - cR_k (the diagonal of T_S)
      const int64_t P2 = sq(P);
      NEGF_TRY(comb(p->r_base[k], P2, &p->r_A[k], 1.0, &p->r_cL[k], -1.0, k + 1 < nd ? &p->r_cR[k] : nullptr, -1.0,
                    nullptr, 0.0));
    }
    // left / right self-energies of every separator on T_S's chain (by
    // sequential sweeps or the recursion), then the connected Green's
    // functions step 4 needs
    NEGF_TRY(chain_solve(0));
    for (int k = 0; k < nd; ++k) {
      const int64_t P2 = sq(p->Psz[k]);
      const negf_plan_s::Reg* LLk = k > 0 ? &p->r_LL[k] : nullptr;
      const negf_plan_s::Reg* RRk = k + 1 < nd ? &p->r_RR[k] : nullptr;
      if (k + 1 < nd) {   // gL at separator k without sub-domain k + 1
        NEGF_TRY(comb(p->r_gLs[k], P2, &p->r_A[k], 1.0, &p->r_cL[k], -1.0, LLk, -1.0, nullptr, 0.0));
        NEGF_TRY(inv_reg(p->r_gLs[k], k));
      }
      if (k > 0) {        // gR at separator k including sub-domain k (the G_1N chain)
        NEGF_TRY(comb(p->r_gRin[k], P2, &p->r_base[k], 1.0, RRk, -1.0, nullptr, 0.0, nullptr, 0.0));
        NEGF_TRY(inv_reg(p->r_gRin[k], k));
      }
      NEGF_TRY(comb(p->r_gRs[k], P2, &p->r_A[k], 1.0, k + 1 < nd ? &p->r_cR[k] : nullptr, -1.0, RRk, -1.0, nullptr, 0.0));
      NEGF_TRY(inv_reg(p->r_gRs[k], k));
      NEGF_TRY(comb(p->r_Gpp[k], P2, &p->r_base[k], 1.0, LLk, -1.0, RRk, -1.0, nullptr, 0.0));
      NEGF_TRY(inv_reg(p->r_Gpp[k], k));
    }
    return cudaSuccess;
  }

  // ---- the interface's chains (Alg. 2 step 3) ----------------------------
  // Chain c: nodes 0..n-1 with diagonal D_k, couplings U_k (k, k+1) and L_k
  // (k+1, k); LL_k = L_{k-1} gL_{k-1} U_{k-1} and RR_k = U_k gR_{k+1} L_k are
  // the node's left / right self-energies, gL / gR the left- / right-connected
  // Green's functions (LL_0 and RR_{n-1} are absent).
  const negf_plan_s::Reg* opt(const std::vector<negf_plan_s::Reg>& v, int k, bool present) const {
    return present ? &v[k] : nullptr;
  }

  // C = alpha A B on node-sized per-energy regions (FP64).
  cudaError_t mmr(int m, int n, int k, const negf_plan_s::Reg& A, const negf_plan_s::Reg& B,
                  const negf_plan_s::Reg& Cr, double alpha, const negf_plan_s::Reg* C1 = nullptr, double beta1 = 1.0) {
    return mm(0, m, n, k, R(A), A.sz, k, R(B), B.sz, n, R(Cr), Cr.sz, n, alpha, false, C1 ? R(*C1) : nullptr,
              C1 ? C1->sz : 0, n, beta1);
  }
  cudaError_t inv_chain(const negf_plan_s::Reg& src, const negf_plan_s::Reg& dst, int P) {
    return s.inv(R(src), src.sz, R(dst), dst.sz, P, C, 0);
  }

  // Sequential sweeps over chain c (the deepest level).
  cudaError_t chain_sweeps(DDChain& c) {
    const int n = c.n;
    // left: gL_0 = D_0^{-1}; LL_k = L_{k-1} gL_{k-1} U_{k-1}, gL_k = (D_k - LL_k)^{-1}
    NEGF_TRY(inv_chain(c.D[0], c.t[0], c.sz[0]));
    for (int k = 1; k < n; ++k) {
      NEGF_TRY(mmr(c.sz[k], c.sz[k - 1], c.sz[k - 1], c.L[k - 1], c.t[k - 1], c.tmp[k], 1.0));
      NEGF_TRY(mmr(c.sz[k], c.sz[k], c.sz[k - 1], c.tmp[k], c.U[k - 1], c.LL[k], 1.0));
      if (k + 1 < n) {
        NEGF_TRY(comb(c.t[k], sq(c.sz[k]), &c.D[k], 1.0, &c.LL[k], -1.0, nullptr, 0.0, nullptr, 0.0));
        NEGF_TRY(inv_chain(c.t[k], c.t[k], c.sz[k]));
      }
    }
    // right: gR_{n-1} = D_{n-1}^{-1}; RR_k = U_k gR_{k+1} L_k, gR_k = (D_k - RR_k)^{-1}
    NEGF_TRY(inv_chain(c.D[n - 1], c.t[n - 1], c.sz[n - 1]));
    for (int k = n - 2; k >= 0; --k) {
      NEGF_TRY(mmr(c.sz[k], c.sz[k + 1], c.sz[k + 1], c.U[k], c.t[k + 1], c.tmp[k], 1.0));
      NEGF_TRY(mmr(c.sz[k], c.sz[k], c.sz[k + 1], c.tmp[k], c.L[k], c.RR[k], 1.0));
      if (k > 0) {
        NEGF_TRY(comb(c.t[k], sq(c.sz[k]), &c.D[k], 1.0, &c.RR[k], -1.0, nullptr, 0.0, nullptr, 0.0));
        NEGF_TRY(inv_chain(c.t[k], c.t[k], c.sz[k]));
      }
    }
    return cudaSuccess;
  }

  // Step 1 on chain c, pair J: corners of the closed group [f, l]: X_FF = t_f
  // of the right-connected sweep, X_FL / X_LF from its first row / column,
  // X_LL from the left-connected sweep.
  double2* ring(const negf_plan_s::Reg& r, int slot, int64_t slot_elems) const { return R(r) + slot * slot_elems; }
  cudaError_t chain_corners(DDChain& c, int J) {
    const int f = c.f[J], l = c.l[J], Ff = c.sz[f];
    NEGF_TRY(cp(R(c.D[l]), c.D[l].sz, c.sz[l], R(c.s1[J]), c.s1[J].sz, c.sz[l], c.sz[l], c.sz[l], 1.0, 0, C));
    for (int k = l; k >= f; --k) {
      NEGF_TRY(inv_chain(c.s1[J], c.t[k], c.sz[k]));
      if (k == f) break;
      const int Bp = c.sz[k - 1], B = c.sz[k];
      NEGF_TRY(mmr(Bp, B, B, c.U[k - 1], c.t[k], c.Y[k], 1.0));      // Y_k = U_{k-1} t_k
      NEGF_TRY(mmr(B, Bp, B, c.t[k], c.L[k - 1], c.X[k], 1.0));      // X_k = t_k L_{k-1}
      NEGF_TRY(mm(0, Bp, Bp, B, R(c.Y[k]), c.Y[k].sz, B, R(c.L[k - 1]), c.L[k - 1].sz, Bp, R(c.s1[J]), c.s1[J].sz, Bp,
                  -1.0, false, R(c.D[k - 1]), c.D[k - 1].sz, Bp, 1.0));   // S_{k-1} = D_{k-1} - Y_k L_{k-1}
    }
    const int64_t sr = (int64_t)Ff * p->Pmax;
    for (int k = f + 1; k <= l; ++k) {   // X_{F,k} = -X_{F,k-1} Y_k, X_{k,F} = -X_k X_{k-1,F}
      const int B = c.sz[k], Bp = c.sz[k - 1];
      const double2* rp = k - 1 == f ? R(c.t[f]) : ring(c.row[J], (k - 1) & 1, sr);
      const int64_t srp = k - 1 == f ? c.t[f].sz : c.row[J].sz;
      NEGF_TRY(mm(0, Ff, B, Bp, rp, srp, Bp, R(c.Y[k]), c.Y[k].sz, B, ring(c.row[J], k & 1, sr), c.row[J].sz, B, -1.0));
      const double2* cpv = k - 1 == f ? R(c.t[f]) : ring(c.col[J], (k - 1) & 1, sr);
      const int64_t scp = k - 1 == f ? c.t[f].sz : c.col[J].sz;
      NEGF_TRY(mm(0, B, Ff, Bp, R(c.X[k]), c.X[k].sz, Bp, cpv, scp, Ff, ring(c.col[J], k & 1, sr), c.col[J].sz, Ff, -1.0));
    }
    // left-connected sweep: X_LL
    NEGF_TRY(cp(R(c.D[f]), c.D[f].sz, Ff, R(c.s1[J]), c.s1[J].sz, Ff, Ff, Ff, 1.0, 0, C));
    for (int k = f; k <= l; ++k) {
      if (k == l) return inv_chain(c.s1[J], c.xll[J], c.sz[k]);
      NEGF_TRY(inv_chain(c.s1[J], c.s2[J], c.sz[k]));
      const int B = c.sz[k], Bn = c.sz[k + 1];
      NEGF_TRY(mm(0, Bn, B, B, R(c.L[k]), c.L[k].sz, B, R(c.s2[J]), c.s2[J].sz, B, R(c.tmp[k]), c.tmp[k].sz, B, 1.0));
      NEGF_TRY(mm(0, Bn, Bn, B, R(c.tmp[k]), c.tmp[k].sz, B, R(c.U[k]), c.U[k].sz, Bn, R(c.s1[J]), c.s1[J].sz, Bn, -1.0,
                  false, R(c.D[k + 1]), c.D[k + 1].sz, Bn, 1.0));
    }
    return cudaSuccess;
  }
  // corners of pair J's group as (pointer, per-energy stride)
  const double2* cXFF(DDChain& c, int J, int64_t* st) { *st = c.t[c.f[J]].sz; return R(c.t[c.f[J]]); }
  const double2* cXFL(DDChain& c, int J, int64_t* st) {
    const int f = c.f[J], l = c.l[J];
    if (l == f) { *st = c.t[f].sz; return R(c.t[f]); }
    *st = c.row[J].sz;
    return ring(c.row[J], l & 1, (int64_t)c.sz[f] * p->Pmax);
  }
  const double2* cXLF(DDChain& c, int J, int64_t* st) {
    const int f = c.f[J], l = c.l[J];
    if (l == f) { *st = c.t[f].sz; return R(c.t[f]); }
    *st = c.col[J].sz;
    return ring(c.col[J], l & 1, (int64_t)c.sz[f] * p->Pmax);
  }

  // Step 4 on chain c, pair J: the group's left / right self-energies from
  // the separators' (open sweeps with the boundary self-energies).
  cudaError_t chain_open(DDChain& c, int J) {
    const int f = c.f[J], l = c.l[J], q = l + 1;
    if (J > 0) {   // LL_f = L_{f-1} (D_p - LL_p)^{-1} U_{f-1}, p = f - 1
      const int pn = f - 1, P = c.sz[pn];
      NEGF_TRY(comb(c.s2[J], sq(P), &c.D[pn], 1.0, &c.LL[pn], -1.0, nullptr, 0.0, nullptr, 0.0));
      NEGF_TRY(inv_chain(c.s2[J], c.s2[J], P));
      NEGF_TRY(mmr(c.sz[f], P, P, c.L[pn], c.s2[J], c.tmp[f], 1.0));
      NEGF_TRY(mmr(c.sz[f], c.sz[f], P, c.tmp[f], c.U[pn], c.LL[f], 1.0));
    }
    for (int k = f; k <= l; ++k) {   // open left sweep
      if (k > f) {
        NEGF_TRY(mmr(c.sz[k], c.sz[k - 1], c.sz[k - 1], c.L[k - 1], c.s1[J], c.tmp[k], 1.0));
        NEGF_TRY(mmr(c.sz[k], c.sz[k], c.sz[k - 1], c.tmp[k], c.U[k - 1], c.LL[k], 1.0));
      }
      if (k == l) break;
      NEGF_TRY(comb(c.s1[J], sq(c.sz[k]), &c.D[k], 1.0, opt(c.LL, k, k > 0), -1.0, nullptr, 0.0, nullptr, 0.0));
      NEGF_TRY(inv_chain(c.s1[J], c.s1[J], c.sz[k]));
    }
    {   // RR_l = U_l (D_q - RR_q)^{-1} L_l
      const int P = c.sz[q];
      NEGF_TRY(comb(c.s2[J], sq(P), &c.D[q], 1.0, opt(c.RR, q, q + 1 < c.n), -1.0, nullptr, 0.0, nullptr, 0.0));
      NEGF_TRY(inv_chain(c.s2[J], c.s2[J], P));
      NEGF_TRY(mmr(c.sz[l], P, P, c.U[l], c.s2[J], c.tmp[l], 1.0));
      NEGF_TRY(mmr(c.sz[l], c.sz[l], P, c.tmp[l], c.L[l], c.RR[l], 1.0));
    }
    for (int k = l; k >= f; --k) {   // open right sweep
      if (k < l) {
        NEGF_TRY(mmr(c.sz[k], c.sz[k + 1], c.sz[k + 1], c.U[k], c.s1[J], c.tmp[k], 1.0));
        NEGF_TRY(mmr(c.sz[k], c.sz[k], c.sz[k + 1], c.tmp[k], c.L[k], c.RR[k], 1.0));
      }
      if (k == f) break;
      NEGF_TRY(comb(c.s1[J], sq(c.sz[k]), &c.D[k], 1.0, &c.RR[k], -1.0, nullptr, 0.0, nullptr, 0.0));
      NEGF_TRY(inv_chain(c.s1[J], c.s1[J], c.sz[k]));
    }
    return cudaSuccess;
  }

  // Left / right self-energies of every node of chain ci.
  cudaError_t chain_solve(int ci) {
    if (p->chains[ci].child < 0) return chain_sweeps(p->chains[ci]);
    const int np = p->chains[ci].np;
    NEGF_TRY(for_count(np, [&](DD& d, int J) { return d.chain_corners(d.p->chains[ci], J); }));
    {   // the next level's chain over this level's separators
      DDChain& c = p->chains[ci];
      DDChain& h = p->chains[c.child];
      for (int J = 0; J < np; ++J) {
        const int q = c.l[J] + 1, P = c.sz[q], lq = c.l[J], Pl = c.sz[lq];
        // cL_q = L_{l} X_LL U_{l} (the group left of q)
        NEGF_TRY(mmr(P, Pl, Pl, c.L[lq], c.xll[J], c.tmp[q], 1.0));
        NEGF_TRY(mmr(P, P, Pl, c.tmp[q], c.U[lq], c.cL[q], 1.0));
        const negf_plan_s::Reg* cRq = nullptr;
        if (J + 1 < np) {   // the group right of q: cR_q, and the couplings to the next separator
          const int f1 = c.f[J + 1], l1 = c.l[J + 1], F = c.sz[f1], Ln = c.sz[l1], q1 = l1 + 1, P1 = c.sz[q1];
          int64_t sff = 0, sfl = 0, slf = 0;
          const double2* xff = cXFF(c, J + 1, &sff);
          const double2* xfl = cXFL(c, J + 1, &sfl);
          const double2* xlf = cXLF(c, J + 1, &slf);
          NEGF_TRY(mm(0, P, F, F, R(c.U[q]), c.U[q].sz, F, xff, sff, F, R(c.tmp[q]), c.tmp[q].sz, F, 1.0));
          NEGF_TRY(mm(0, P, P, F, R(c.tmp[q]), c.tmp[q].sz, F, R(c.L[q]), c.L[q].sz, P, R(c.cR[q]), c.cR[q].sz, P, 1.0));
          cRq = &c.cR[q];
          // U'_J = -U_q X_FL U_{l1},  L'_J = -L_{l1} X_LF L_q
          NEGF_TRY(mm(0, P, Ln, F, R(c.U[q]), c.U[q].sz, F, xfl, sfl, Ln, R(c.tmp[q]), c.tmp[q].sz, Ln, 1.0));
          NEGF_TRY(mm(0, P, P1, Ln, R(c.tmp[q]), c.tmp[q].sz, Ln, R(c.U[l1]), c.U[l1].sz, P1, R(h.U[J]), h.U[J].sz, P1,
                      -1.0));
          NEGF_TRY(mm(0, P1, F, Ln, R(c.L[l1]), c.L[l1].sz, Ln, xlf, slf, F, R(c.tmp[q1]), c.tmp[q1].sz, F, 1.0));
          NEGF_TRY(mm(0, P1, P, F, R(c.tmp[q1]), c.tmp[q1].sz, F, R(c.L[q]), c.L[q].sz, P, R(h.L[J]), h.L[J].sz, P,
                      -1.0));
        }
        NEGF_TRY(comb(h.D[J], sq(P), &c.D[q], 1.0, &c.cL[q], -1.0, cRq, -1.0, nullptr, 0.0));
      }
    }
    NEGF_TRY(chain_solve(p->chains[ci].child));
    {   // the separators' self-energies: the adjacent groups plus the next level's
      DDChain& c = p->chains[ci];
      DDChain& h = p->chains[c.child];
      for (int J = 0; J < np; ++J) {
        const int q = c.l[J] + 1;
        const int64_t P2 = sq(c.sz[q]);
        NEGF_TRY(comb(c.LL[q], P2, &c.cL[q], 1.0, J > 0 ? &h.LL[J] : nullptr, 1.0, nullptr, 0.0, nullptr, 0.0));
        if (J + 1 < np)
          NEGF_TRY(comb(c.RR[q], P2, &c.cR[q], 1.0, &h.RR[J], 1.0, nullptr, 0.0, nullptr, 0.0));
      }
    }
    return for_count(np, [&](DD& d, int J) { return d.chain_open(d.p->chains[ci], J); });
  }

  // Step 4 for domain j: boundary self-energies, the open sub-domain's RGF
  // into the band, and the band blocks between the sub-domain and its
  // separators.  For j = 0 with want_row, also G_{1,P_0} (into r_g1 slot 0).
  cudaError_t open_domain(int j, bool want_row) {
    const int f = p->dom_f[j], l = p->dom_l[j], F = p->Fsz[j], L = p->Lsz[j], P = p->Psz[j];
    const int P0 = j > 0 ? p->Psz[j - 1] : 0;
    double2* WR = R(p->r_wr[j]);
    double2* VR = R(p->r_vr[j]);
    double2* SR = R(p->r_sr[j]);
    const int64_t sWR = p->r_wr[j].sz, sVR = p->r_vr[j].sz, sSR = p->r_sr[j].sz;
    // W_R = M_{L,P} gR_P, V_R = gR_P M_{P,L}, Sigma_right = W_R M_{P,L}
    NEGF_TRY(mm(0, L, P, P, HF(p->mlq_off[j]), 0, P, R(p->r_gRs[j]), p->r_gRs[j].sz, P, WR, sWR, P, 1.0));
    NEGF_TRY(mm(0, P, L, P, R(p->r_gRs[j]), p->r_gRs[j].sz, P, HF(p->mql_off[j]), 0, L, VR, sVR, L, 1.0));
    NEGF_TRY(mm(0, L, L, P, WR, sWR, P, HF(p->mql_off[j]), 0, L, SR, sSR, L, 1.0));
    double2 *WL = nullptr, *VL = nullptr, *SL = nullptr;
    const int64_t sWL = p->r_wl[j].sz, sVL = p->r_vl[j].sz, sSL = p->r_sl[j].sz;
    if (j > 0) {   // W_L = M_{F,p} gL_p, V_L = gL_p M_{p,F}, Sigma_left = W_L M_{p,F}
      WL = R(p->r_wl[j]); VL = R(p->r_vl[j]); SL = R(p->r_sl[j]);
      NEGF_TRY(mm(0, F, P0, P0, HF(p->mfp_off[j]), 0, P0, R(p->r_gLs[j - 1]), p->r_gLs[j - 1].sz, P0, WL, sWL, P0, 1.0));
      NEGF_TRY(mm(0, P0, F, P0, R(p->r_gLs[j - 1]), p->r_gLs[j - 1].sz, P0, HF(p->mpf_off[j]), 0, F, VL, sVL, F, 1.0));
      NEGF_TRY(mm(0, F, F, P0, WL, sWL, P0, HF(p->mpf_off[j]), 0, F, SL, sSL, F, 1.0));
    }
    s.xr = SR; s.xr_s = sSR; s.xr_ld = L; s.xr_f = l - w + 1;
    s.xl = SL; s.xl_s = sSL; s.xl_ld = F; s.xl_f = j > 0 ? f : -1;
    NEGF_TRY(s.upward(true, f, l));
    NEGF_TRY(s.downward(f, l));
    s.xr = s.xl = nullptr;
    // blocks between L and the right separator:
    //   G_{a,s} = -sum_{c in L} G_{a,c} W_R[c, s],  G_{s,a} = -sum_{c in L} V_R[s, c] G_{c,a}
    for (int a = l - w + 1; a <= l; ++a)
      for (int sl = l + 1; sl <= l + w; ++sl) {
        if (sl - a > w) continue;
        bool first = true;
        for (int c = l - w + 1; c <= l; ++c) {
          NEGF_TRY(mm(1, b(a), b(sl), b(c), s.Gb(a, c), sG, b(c), WR + (int64_t)offL(c) * P + p->off_in[sl], sWR, P,
                      s.Gb(a, sl), sG, b(sl), -1.0, !first));
          NEGF_TRY(mm(1, b(sl), b(a), b(c), VR + (int64_t)p->off_in[sl] * L + offL(c), sVR, L, s.Gb(c, a), sG, b(a),
                      s.Gb(sl, a), sG, b(a), -1.0, !first));
          first = false;
        }
      }
    if (j > 0)   // blocks between F and the left separator
      for (int a = f; a < f + w; ++a)
        for (int sl = f - w; sl < f; ++sl) {
          if (a - sl > w) continue;
          bool first = true;
          for (int c = f; c < f + w; ++c) {
            NEGF_TRY(mm(1, b(a), b(sl), b(c), s.Gb(a, c), sG, b(c), WL + (int64_t)offF(c) * P0 + p->off_in[sl], sWL, P0,
                        s.Gb(a, sl), sG, b(sl), -1.0, !first));
            NEGF_TRY(mm(1, b(sl), b(a), b(c), VL + (int64_t)p->off_in[sl] * F + offF(c), sVL, F, s.Gb(c, a), sG, b(a),
                        s.Gb(sl, a), sG, b(a), -1.0, !first));
            first = false;
          }
        }
    if (j == 0 && want_row) {
      // first row inside D2_0 (Eq. 4x4_exact_RGF first row, with this
      // sub-domain's open multipliers), then G_{1,P_0} = -sum_{c in L} G_{1,c} W_R[c, :]
      const int b0 = b(0);
      NEGF_TRY(s.misc([&] { return negf::copy_blocks(s.Tblk(0), sq(b0), s.Rblk(0), s.sR(0), sq(b0), C, s.st); }));
      for (int jj = 1; jj <= l; ++jj) {
        const int lo = std::max(0, jj - w);
        for (int c = lo; c < jj; ++c)
          NEGF_TRY(mm(1, b0, b(jj), b(c), s.Rblk(c), s.sR(c), b(c), s.Yblk(c, jj), (int64_t)b(c) * b(jj), b(jj),
                      s.Rblk(jj), s.sR(jj), b(jj), -1.0, c > lo));
      }
      double2* g0 = R(p->r_g1);
      const int64_t sg = p->r_g1.sz;
      bool first = true;
      for (int c = l - w + 1; c <= l; ++c) {
        NEGF_TRY(mm(1, b0, P, b(c), s.Rblk(c), s.sR(c), b(c), WR + (int64_t)offL(c) * P, sWR, P, g0, sg, P, -1.0, !first));
        first = false;
      }
    }
    return cudaSuccess;
  }

  // Separator band blocks from the diagonals of T_S^{-1}.
  cudaError_t separators() {
    for (int k = 0; k < nd; ++k) {
      const int P = p->Psz[k], s0 = p->dom_l[k] + 1;
      for (int a = s0; a < s0 + w; ++a)
        for (int c = s0; c < s0 + w; ++c)
          NEGF_TRY(cp(R(p->r_Gpp[k]) + (int64_t)p->off_in[a] * P + p->off_in[c], p->r_Gpp[k].sz, P, s.Gb(a, c), sG, b(c),
                      b(a), b(c), 1.0, 0, C));
    }
    return cudaSuccess;
  }

  // G_1N: G_{1,P_k} = -G_{1,P_{k-1}} T_S[k-1,k] gR_k through the separators
  // (first-row relation of the chain reduced to D2_0 and the separators),
  // then the columns of layer N.
  cudaError_t g1n(double2* out, int64_t sOut) {
    const int N = p->N, b0 = b(0);
    const int64_t slot = (int64_t)b0 * p->Pmax, sg = p->r_g1.sz;
    double2* base = R(p->r_g1);
    double2* T = R(p->r_g1t);
    int cur = 0;
    for (int k = 1; k < nd; ++k) {
      const int Pm = p->Psz[k - 1], P = p->Psz[k];
      NEGF_TRY(mm(0, b0, P, Pm, base + cur * slot, sg, Pm, R(p->r_Tu[k - 1]), p->r_Tu[k - 1].sz, P, T, p->r_g1t.sz, P, 1.0));
      NEGF_TRY(mm(0, b0, P, P, T, p->r_g1t.sz, P, R(p->r_gRin[k]), p->r_gRin[k].sz, P, base + (1 - cur) * slot, sg, P,
                  -1.0));
      cur = 1 - cur;
    }
    const int Pn = p->Psz[nd - 1];
    return cp(base + cur * slot + p->off_in[N - 1], sg, Pn, out, sOut, b(N - 1), b0, b(N - 1), 1.0, 0, C);
  }

  // Runs f(dd_j, j) for every sub-domain j concurrently: domain j of this
  // energy group on its own stream (graph branch), joined back afterwards.
  // Each domain sweeps in its own Schur-window slots; everything else a
  // domain writes is disjoint from the other domains'.
  template <class F>
  cudaError_t for_domains(F f) { return for_count(nd, f); }

  // Runs f(dd_j, j) for j < cnt (cnt <= n_domains) on the group's domain
  // streams, concurrently, joined back afterwards.
  template <class F>
  cudaError_t for_count(int cnt, F f) {
    const int g = s.grp;
    NEGF_TRY(cudaEventRecord(p->dfork[g], s.st));
    for (int j = 1; j < cnt; ++j) NEGF_TRY(cudaStreamWaitEvent(p->dstream[(size_t)g * nd + j], p->dfork[g], 0));
    for (int j = 0; j < cnt; ++j) {
      Sweep sj = s;
      sj.sdom = j;
      if (j > 0) {
        sj.st = p->dstream[(size_t)g * nd + j];
        sj.after_first_inv = nullptr;
      }
      DD dj(p, sj);
      NEGF_TRY(f(dj, j));
      if (j == 0) s.after_first_inv = sj.after_first_inv;
    }
    for (int j = 1; j < cnt; ++j) {
      NEGF_TRY(cudaEventRecord(p->djoin[(size_t)g * nd + j], p->dstream[(size_t)g * nd + j]));
      NEGF_TRY(cudaStreamWaitEvent(s.st, p->djoin[(size_t)g * nd + j], 0));
    }
    return cudaSuccess;
  }

  cudaError_t run(bool want_band, double2* g1n_out, int64_t s1) {
    NEGF_TRY(for_domains([&](DD& d, int j) { return d.corners(j); }));
    NEGF_TRY(interface());
    if (want_band) {
      NEGF_TRY(for_domains([&](DD& d, int j) { return d.open_domain(j, j == 0 && g1n_out != nullptr); }));
      NEGF_TRY(separators());
    } else {
      NEGF_TRY(open_domain(0, true));
    }
    if (g1n_out) NEGF_TRY(g1n(g1n_out, s1));
    return cudaSuccess;
  }
};

}  // namespace
