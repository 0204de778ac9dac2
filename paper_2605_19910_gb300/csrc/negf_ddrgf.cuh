// DDRGF (Sec. 3, Alg. 2) schedule of one energy range (one TU: included by
// negf_capi.cu only).
#pragma once

#include "negf_sweep.cuh"

namespace {

// ---------------------------------------------------------------------------
// DDRGF (Sec. 3, Alg. 2) for one energy range: per-domain extended RGF,
// the interface Schur complement T_S in FP64, its block tridiagonal RGF
// (Prop. 4) in FP64, and the stitching of the four parts of
// Eq. 2x2_explicit_inverse_parallel_DDRGF restricted to the band.
// ---------------------------------------------------------------------------
struct DD {
  negf_plan_s* p;
  Sweep& s;
  int w, nd, C;
  int64_t sG;

  DD(negf_plan_s* pp, Sweep& ss) : p(pp), s(ss), w(pp->w), nd(pp->n_domains), C(ss.ne), sG(pp->band_elems) {}

  int b(int i) const { return p->b[i]; }
  int Pp(int j) const { return j > 0 ? p->Psz[j - 1] : 0; }
  double2* reg(double2* base, int64_t off, int64_t size) const {
    return base + off * p->chunk + (int64_t)s.wofs * size;
  }
  int offF(int c) const {          // column offset of layer c inside F of its domain
    const int j = p->dom_of[c];
    int o = 0;
    for (int k = p->dom_f[j]; k < c; ++k) o += b(k);
    return o;
  }
  int offL(int c) const {          // column offset of layer c inside Lw of its domain
    const int j = p->dom_of[c];
    int o = 0;
    for (int k = p->dom_l[j] - w + 1; k < c; ++k) o += b(k);
    return o;
  }
  bool inF(int c) const { const int j = p->dom_of[c]; return j >= 0 && c < p->dom_f[j] + w; }
  bool inL(int c) const { const int j = p->dom_of[c]; return j >= 0 && c > p->dom_l[j] - w; }
  int Fj(int a) const { return p->Fsz[p->dom_of[a]]; }
  int Lj(int a) const { return p->Lsz[p->dom_of[a]]; }
  int Pj(int a) const { return p->Psz[p->dom_of[a]]; }
  int Pm(int a) const { return Pp(p->dom_of[a]); }

  double2* FC(int a) const { return reg(p->FC, p->fc_off[a], (int64_t)b(a) * Fj(a)); }
  double2* FR(int a) const { return reg(p->FR, p->fc_off[a], (int64_t)b(a) * Fj(a)); }
  double2* LC(int a) const { return reg(p->LCd, p->lc_off[a], (int64_t)b(a) * Lj(a)); }
  double2* LR(int a) const { return reg(p->LR, p->lc_off[a], (int64_t)b(a) * Lj(a)); }
  double2* VT(int a) const { return reg(p->VT, p->lc_off[a], (int64_t)b(a) * Lj(a)); }
  double2* Wp(int a) const { return reg(p->Wp, p->wp_off[a], (int64_t)b(a) * Pm(a)); }
  double2* Vp(int a) const { return reg(p->Vp, p->wp_off[a], (int64_t)b(a) * Pm(a)); }
  double2* Zp(int a) const { return reg(p->Zp, p->wp_off[a], (int64_t)b(a) * Pm(a)); }
  double2* Wq(int a) const { return reg(p->Wq, p->wq_off[a], (int64_t)b(a) * Pj(a)); }
  double2* Vq(int a) const { return reg(p->Vq, p->wq_off[a], (int64_t)b(a) * Pj(a)); }
  double2* Zq(int a) const { return reg(p->Zq, p->wq_off[a], (int64_t)b(a) * Pj(a)); }
  double2* TSd(int k) const { return reg(p->TSd, p->tsd_off[k], sq(p->Psz[k])); }
  double2* GSd(int k) const { return reg(p->GSd, p->tsd_off[k], sq(p->Psz[k])); }
  double2* tS(int k) const { return reg(p->tS, p->tsd_off[k], sq(p->Psz[k])); }
  double2* TSu(int k) const { return reg(p->TSu, p->tsu_off[k], (int64_t)p->Psz[k] * p->Psz[k + 1]); }
  double2* TSl(int k) const { return reg(p->TSl, p->tsu_off[k], (int64_t)p->Psz[k] * p->Psz[k + 1]); }
  double2* GSu(int k) const { return reg(p->GSu, p->tsu_off[k], (int64_t)p->Psz[k] * p->Psz[k + 1]); }
  double2* GSl(int k) const { return reg(p->GSl, p->tsu_off[k], (int64_t)p->Psz[k] * p->Psz[k + 1]); }
  double2* XS(int k) const { return reg(p->XS, p->ts_x_off[k], (int64_t)p->Psz[k] * p->Psz[k - 1]); }
  double2* YS(int k) const { return reg(p->YS, p->ts_x_off[k], (int64_t)p->Psz[k] * p->Psz[k - 1]); }
  double2* RS(int k) const { return reg(p->RS, p->rs_off[k], (int64_t)p->Psz[0] * p->Psz[k]); }
  double2* SS() const { return reg(p->SS, 0, sq(p->Pmax)); }

  // C (+)= alpha A B with per-energy strides (0 = shared operand);
  // lowp routes through the plan's precision, otherwise FP64.
  cudaError_t mm(bool lowp, int m, int n, int k, const double2* A, int64_t sA, int lda, const double2* B,
                 int64_t sB, int ldb, double2* Cm, int64_t sC, int ldc, double alpha, bool acc,
                 const double2* C1 = nullptr, int64_t sC1 = 0, int ldc1 = 0) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    ZGemm g;
    g.m = m; g.n = n; g.k = k;
    g.A = A; g.sA = sA; g.lda = lda;
    g.B = B; g.sB = sB; g.ldb = ldb;
    g.C = Cm; g.sC = sC; g.ldc = ldc;
    g.alpha = {alpha, 0.0};
    if (C1) { g.C1 = C1; g.sC1 = sC1; g.ldc1 = ldc1; g.beta1 = {1.0, 0.0}; }
    else if (acc) { g.C1 = Cm; g.sC1 = sC; g.ldc1 = ldc; g.beta1 = {1.0, 0.0}; }
    g.batch = C;
    return lowp ? s.gemm(g) : s.gemm64(g);
  }
  cudaError_t cp(const double2* src, int64_t sSrc, int ldSrc, double2* dst, int64_t sDst, int ldDst, int rows,
                 int cols, double scale, int acc, int batch) {
    return s.misc([&] { return negf::copy2d(src, sSrc, ldSrc, dst, sDst, ldDst, rows, cols, scale, acc, batch, s.st); });
  }
  cudaError_t eye(double2* dst, int64_t sDst, int ld, int rows, int cols, int off, int nid, int rows_mode, int batch) {
    return s.misc([&] { return negf::set_eye(dst, sDst, ld, rows, cols, off, nid, rows_mode, batch, s.st); });
  }

  // Energy-independent super-blocks of M = -H between a domain's first /
  // last w layers and its separators.
  cudaError_t assemble_msup() {
    for (int j = 0; j < nd; ++j) {
      const int f = p->dom_f[j], l = p->dom_l[j], F = p->Fsz[j], L = p->Lsz[j], P = p->Psz[j], P0 = Pp(j);
      double2* MFp = p->Msup + p->mfp_off[j];
      double2* MpF = p->Msup + p->mpf_off[j];
      double2* MLq = p->Msup + p->mlq_off[j];
      double2* MqL = p->Msup + p->mql_off[j];
      NEGF_TRY(eye(MLq, 0, P, L, P, 0, 0, 0, 1));
      NEGF_TRY(eye(MqL, 0, L, P, L, 0, 0, 0, 1));
      if (P0) {
        NEGF_TRY(eye(MFp, 0, P0, F, P0, 0, 0, 0, 1));
        NEGF_TRY(eye(MpF, 0, F, P0, F, 0, 0, 0, 1));
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

  // Step 1 of Alg. 2 for domain j: X = (M restricted to D2_j)^{-1}, its band
  // (into the band output) and its first / last w block rows and columns
  // (the internal halos of Sec. 3, "Data dependencies").
  cudaError_t domain(int j) {
    const int f = p->dom_f[j], l = p->dom_l[j], F = p->Fsz[j], L = p->Lsz[j];
    NEGF_TRY(s.upward(true, f, l));
    NEGF_TRY(s.downward(f, l));
    // First w columns: X_{i,c} = -sum_{c'} Xm_{i,c'} X_{c',c}  (i > c), band values elsewhere.
    for (int i = f; i <= l; ++i) {
      const int lo = std::max(f, i - w);
      for (int c = lo; c < i; ++c)
        NEGF_TRY(mm(true, b(i), F, b(c), s.Xblk(i, c), (int64_t)b(i) * b(c), b(c), FC(c), (int64_t)b(c) * F, F,
                    FC(i), (int64_t)b(i) * F, F, -1.0, c > lo));
      for (int c = f; c < f + w; ++c)
        if (c >= i) NEGF_TRY(cp(s.Gb(i, c), sG, b(c), FC(i) + offF(c), (int64_t)b(i) * F, F, b(i), b(c), 1.0, 0, C));
    }
    // First w rows: X_{c,j'} = -sum_{c'} X_{c,c'} Y_{c',j'}  (j' > c), band values elsewhere.
    for (int jj = f; jj <= l; ++jj) {
      const int lo = std::max(f, jj - w);
      for (int c = lo; c < jj; ++c)
        NEGF_TRY(mm(true, F, b(jj), b(c), FR(c), (int64_t)b(c) * F, b(c), s.Yblk(c, jj), (int64_t)b(c) * b(jj), b(jj),
                    FR(jj), (int64_t)b(jj) * F, b(jj), -1.0, c > lo));
      for (int r = f; r < f + w; ++r)
        if (r >= jj) NEGF_TRY(cp(s.Gb(r, jj), sG, b(jj), FR(jj) + (int64_t)offF(r) * b(jj), (int64_t)b(jj) * F, b(jj),
                                b(r), b(jj), 1.0, 0, C));
    }
    // Last w columns: with M_D = U D L from the upward pass, X E_L =
    // L^{-1} D^{-1} U^{-1} E_L: backward v = U^{-1} E_L, then forward.
    for (int i = l; i >= f; --i) {
      NEGF_TRY(eye(VT(i), (int64_t)b(i) * L, L, b(i), L, inL(i) ? offL(i) : 0, inL(i) ? b(i) : 0, 0, C));
      for (int c = i + 1; c <= std::min(l, i + w); ++c)
        NEGF_TRY(mm(true, b(i), L, b(c), s.Yblk(i, c), (int64_t)b(i) * b(c), b(c), VT(c), (int64_t)b(c) * L, L,
                    VT(i), (int64_t)b(i) * L, L, -1.0, true));
    }
    for (int i = f; i <= l; ++i) {
      NEGF_TRY(mm(true, b(i), L, b(i), s.Tblk(i), sq(b(i)), b(i), VT(i), (int64_t)b(i) * L, L, LC(i),
                  (int64_t)b(i) * L, L, 1.0, false));
      for (int c = std::max(f, i - w); c < i; ++c)
        NEGF_TRY(mm(true, b(i), L, b(c), s.Xblk(i, c), (int64_t)b(i) * b(c), b(c), LC(c), (int64_t)b(c) * L, L,
                    LC(i), (int64_t)b(i) * L, L, -1.0, true));
    }
    // Last w rows: E_L^T L^{-1} D^{-1} U^{-1}: backward u^T, then forward.
    for (int i = l; i >= f; --i) {
      NEGF_TRY(eye(VT(i), (int64_t)b(i) * L, b(i), L, b(i), inL(i) ? offL(i) : 0, inL(i) ? b(i) : 0, 1, C));
      for (int c = i + 1; c <= std::min(l, i + w); ++c)
        NEGF_TRY(mm(true, L, b(i), b(c), VT(c), (int64_t)b(c) * L, b(c), s.Xblk(c, i), (int64_t)b(c) * b(i), b(i),
                    VT(i), (int64_t)b(i) * L, b(i), -1.0, true));
    }
    for (int i = f; i <= l; ++i) {
      NEGF_TRY(mm(true, L, b(i), b(i), VT(i), (int64_t)b(i) * L, b(i), s.Tblk(i), sq(b(i)), b(i), LR(i),
                  (int64_t)b(i) * L, b(i), 1.0, false));
      for (int c = std::max(f, i - w); c < i; ++c)
        NEGF_TRY(mm(true, L, b(i), b(c), LR(c), (int64_t)b(c) * L, b(c), s.Yblk(c, i), (int64_t)b(c) * b(i), b(i),
                    LR(i), (int64_t)b(i) * L, b(i), -1.0, true));
    }
    // W_a = [X_{a,F} M_{F,p}, X_{a,L} M_{L,q}],  V_a = [M_{p,F} X_{F,a}; M_{q,L} X_{L,a}]
    const int P = p->Psz[j], P0 = Pp(j);
    const double2* MFp = p->Msup + p->mfp_off[j];
    const double2* MpF = p->Msup + p->mpf_off[j];
    const double2* MLq = p->Msup + p->mlq_off[j];
    const double2* MqL = p->Msup + p->mql_off[j];
    for (int a = f; a <= l; ++a) {
      NEGF_TRY(mm(true, b(a), P, L, LC(a), (int64_t)b(a) * L, L, MLq, 0, P, Wq(a), (int64_t)b(a) * P, P, 1.0, false));
      NEGF_TRY(mm(true, P, b(a), L, MqL, 0, L, LR(a), (int64_t)b(a) * L, b(a), Vq(a), (int64_t)b(a) * P, b(a), 1.0, false));
      if (P0) {
        NEGF_TRY(mm(true, b(a), P0, F, FC(a), (int64_t)b(a) * F, F, MFp, 0, P0, Wp(a), (int64_t)b(a) * P0, P0, 1.0, false));
        NEGF_TRY(mm(true, P0, b(a), F, MpF, 0, F, FR(a), (int64_t)b(a) * F, b(a), Vp(a), (int64_t)b(a) * P0, b(a), 1.0, false));
      }
    }
    return cudaSuccess;
  }

  // Step 2 (Eq. Schur_complement_in_parallel_DDRGF): T_S = T11 - T12 X T21,
  // block tridiagonal over the separators (Prop. 4), in FP64.
  cudaError_t schur() {
    const int N = p->N;
    for (int k = 0; k < nd; ++k) {
      const int P = p->Psz[k], s0 = p->dom_l[k] + 1;
      NEGF_TRY(eye(TSd(k), sq(P), P, P, P, 0, 0, 0, C));
      for (int a = s0; a < s0 + w; ++a)
        for (int c = s0; c < s0 + w; ++c)
          NEGF_TRY(cp(s.Hblk(a, c), 0, b(c), TSd(k) + (int64_t)p->off_in[a] * P + p->off_in[c], sq(P), P, b(a), b(c),
                      -1.0, 0, C));
      NEGF_TRY(s.misc([&] { return negf::add_diag(TSd(k), sq(P), P, P, s.E + s.e0, 1, 1.0, C, s.st); }));
      if (s0 + w - 1 == N - 1 && s.sigR) {
        const int sl = N - 1;
        NEGF_TRY(cp(s.sigmaR(), s.sig_stride, b(sl), TSd(k) + (int64_t)p->off_in[sl] * P + p->off_in[sl], sq(P), P,
                    b(sl), b(sl), -1.0, 1, C));
      }
      // - M[p_k, L_k] X^(k)[L_k, L_k] M[L_k, p_k]
      const int Lk = p->Lsz[k];
      const double2* MqL = p->Msup + p->mql_off[k];
      for (int r = p->dom_l[k] - w + 1; r <= p->dom_l[k]; ++r)
        NEGF_TRY(mm(false, P, P, b(r), MqL + offL(r), 0, Lk, Wq(r), (int64_t)b(r) * P, P, TSd(k), sq(P), P, -1.0, true));
      if (k + 1 < nd) {
        const int j = k + 1, F = p->Fsz[j], L = p->Lsz[j], P1 = p->Psz[j];
        const double2* MpF = p->Msup + p->mpf_off[j];
        const double2* MqL1 = p->Msup + p->mql_off[j];
        bool first_u = true, first_l = true;
        for (int r = p->dom_f[j]; r < p->dom_f[j] + w; ++r) {
          // - M[p_k, F] X[F, F] M[F, p_k]  and  T_S[p_k, p_{k+1}] = - M[p_k, F] X[F, L] M[L, p_{k+1}]
          NEGF_TRY(mm(false, P, P, b(r), MpF + offF(r), 0, F, Wp(r), (int64_t)b(r) * P, P, TSd(k), sq(P), P, -1.0, true));
          NEGF_TRY(mm(false, P, P1, b(r), MpF + offF(r), 0, F, Wq(r), (int64_t)b(r) * P1, P1, TSu(k),
                      (int64_t)P * P1, P1, -1.0, !first_u));
          first_u = false;
        }
        for (int r = p->dom_l[j] - w + 1; r <= p->dom_l[j]; ++r) {
          // T_S[p_{k+1}, p_k] = - M[p_{k+1}, L] X[L, F] M[F, p_k]
          NEGF_TRY(mm(false, P1, P, b(r), MqL1 + offL(r), 0, L, Wp(r), (int64_t)b(r) * P, P, TSl(k), (int64_t)P * P1, P,
                      -1.0, !first_l));
          first_l = false;
        }
      }
    }
    return cudaSuccess;
  }

  // Step 3: b3diag(T_S^{-1}) by block tridiagonal RGF (Alg. 1) in FP64, and
  // the first super-row of T_S^{-1} when G_1N is wanted.
  cudaError_t interface(bool want_row) {
    const int n = nd;
    const int64_t sSS = sq(p->Pmax);
    NEGF_TRY(cp(TSd(n - 1), sq(p->Psz[n - 1]), p->Psz[n - 1], SS(), sSS, p->Psz[n - 1], p->Psz[n - 1], p->Psz[n - 1],
                1.0, 0, C));
    for (int k = n - 1; k >= 0; --k) {
      const int P = p->Psz[k];
      NEGF_TRY(s.inv(SS(), sSS, tS(k), sq(P), P, C, p->dom_l[k] + 2));
      if (k == 0) break;
      const int P0 = p->Psz[k - 1];
      NEGF_TRY(mm(false, P0, P, P, TSu(k - 1), (int64_t)P0 * P, P, tS(k), sq(P), P, YS(k), (int64_t)P0 * P, P, 1.0, false));
      NEGF_TRY(mm(false, P, P0, P, tS(k), sq(P), P, TSl(k - 1), (int64_t)P0 * P, P0, XS(k), (int64_t)P0 * P, P0, 1.0, false));
      NEGF_TRY(mm(false, P0, P0, P, YS(k), (int64_t)P0 * P, P, TSl(k - 1), (int64_t)P0 * P, P0, SS(), sSS, P0, -1.0, false,
                  TSd(k - 1), sq(P0), P0));
    }
    NEGF_TRY(cp(tS(0), sq(p->Psz[0]), p->Psz[0], GSd(0), sq(p->Psz[0]), p->Psz[0], p->Psz[0], p->Psz[0], 1.0, 0, C));
    for (int k = 1; k < n; ++k) {
      const int P = p->Psz[k], P0 = p->Psz[k - 1];
      NEGF_TRY(mm(false, P0, P, P0, GSd(k - 1), sq(P0), P0, YS(k), (int64_t)P0 * P, P, GSu(k - 1), (int64_t)P0 * P, P,
                  -1.0, false));
      NEGF_TRY(mm(false, P, P0, P0, XS(k), (int64_t)P0 * P, P0, GSd(k - 1), sq(P0), P0, GSl(k - 1), (int64_t)P0 * P, P0,
                  -1.0, false));
      NEGF_TRY(mm(false, P, P, P0, XS(k), (int64_t)P0 * P, P0, GSu(k - 1), (int64_t)P0 * P, P, GSd(k), sq(P), P, -1.0,
                  false, tS(k), sq(P), P));
    }
    if (want_row) {
      const int P0 = p->Psz[0];
      NEGF_TRY(cp(GSd(0), sq(P0), P0, RS(0), sq(P0), P0, P0, P0, 1.0, 0, C));
      for (int k = 1; k < n; ++k) {
        const int P = p->Psz[k], Pq = p->Psz[k - 1];
        NEGF_TRY(mm(false, P0, P, Pq, RS(k - 1), (int64_t)P0 * Pq, Pq, YS(k), (int64_t)Pq * P, P, RS(k), (int64_t)P0 * P,
                    P, -1.0, false));
      }
    }
    return cudaSuccess;
  }

  // Step 4: the band of Eq. 2x2_explicit_inverse_parallel_DDRGF around domain j.
  cudaError_t stitch(int j) {
    const int f = p->dom_f[j], l = p->dom_l[j], P = p->Psz[j], P0 = Pp(j);
    const double2* Gqq = GSd(j);
    const double2* Gpp = j > 0 ? GSd(j - 1) : nullptr;
    const double2* Gpq = j > 0 ? GSu(j - 1) : nullptr;   // P0 x P
    const double2* Gqp = j > 0 ? GSl(j - 1) : nullptr;   // P x P0
    const int64_t sPP = sq(P), sP0 = sq(P0), sX = (int64_t)P0 * P;
    for (int a = f; a <= l; ++a) {   // Z_a = Gamma_S V_a
      NEGF_TRY(mm(true, P, b(a), P, Gqq, sPP, P, Vq(a), (int64_t)b(a) * P, b(a), Zq(a), (int64_t)b(a) * P, b(a), 1.0, false));
      if (P0) {
        NEGF_TRY(mm(true, P, b(a), P0, Gqp, sX, P0, Vp(a), (int64_t)b(a) * P0, b(a), Zq(a), (int64_t)b(a) * P, b(a), 1.0, true));
        NEGF_TRY(mm(true, P0, b(a), P0, Gpp, sP0, P0, Vp(a), (int64_t)b(a) * P0, b(a), Zp(a), (int64_t)b(a) * P0, b(a), 1.0,
                    false));
        NEGF_TRY(mm(true, P0, b(a), P, Gpq, sX, P, Vq(a), (int64_t)b(a) * P, b(a), Zp(a), (int64_t)b(a) * P0, b(a), 1.0, true));
      }
    }
    for (int a = f; a <= l; ++a)     // G_ab = X_ab + W_a Gamma_S V_b
      for (int c = std::max(f, a - w); c <= std::min(l, a + w); ++c) {
        NEGF_TRY(mm(true, b(a), b(c), P, Wq(a), (int64_t)b(a) * P, P, Zq(c), (int64_t)b(c) * P, b(c), s.Gb(a, c), sG, b(c),
                    1.0, true));
        if (P0)
          NEGF_TRY(mm(true, b(a), b(c), P0, Wp(a), (int64_t)b(a) * P0, P0, Zp(c), (int64_t)b(c) * P0, b(c), s.Gb(a, c), sG,
                      b(c), 1.0, true));
      }
    // blocks between the domain and its separators: G_{a,s} = -W_a Gamma_S[:, s], G_{s,a} = -Gamma_S[s, :] V_a
    for (int a = f; a <= l; ++a)
      for (int sl = a - w; sl <= a + w; ++sl) {
        if (sl < 0 || sl >= p->N || p->sep_of[sl] < 0) continue;
        const bool right = p->sep_of[sl] == j;
        const int o = p->off_in[sl];
        // column s of Gamma_S restricted to the q and p super-rows
        const double2* qcol = right ? Gqq + o : Gqp + o;          // q super-row
        const int ldq = right ? P : P0;
        const int64_t sq_ = right ? sPP : sX;
        NEGF_TRY(mm(true, b(a), b(sl), P, Wq(a), (int64_t)b(a) * P, P, qcol, sq_, ldq, s.Gb(a, sl), sG, b(sl), -1.0, false));
        if (P0) {
          const double2* pcol = right ? Gpq + o : Gpp + o;        // p super-row
          const int ldp = right ? P : P0;
          const int64_t sp_ = right ? sX : sP0;
          NEGF_TRY(mm(true, b(a), b(sl), P0, Wp(a), (int64_t)b(a) * P0, P0, pcol, sp_, ldp, s.Gb(a, sl), sG, b(sl), -1.0, true));
        }
        // row s of Gamma_S restricted to the q and p super-columns
        const double2* qrow = right ? Gqq + (int64_t)o * P : Gpq + (int64_t)o * P;
        const int64_t sqr = right ? sPP : sX;
        NEGF_TRY(mm(true, b(sl), b(a), P, qrow, sqr, P, Vq(a), (int64_t)b(a) * P, b(a), s.Gb(sl, a), sG, b(a), -1.0, false));
        if (P0) {
          const double2* prow = right ? Gqp + (int64_t)o * P0 : Gpp + (int64_t)o * P0;
          const int64_t spr = right ? sX : sP0;
          NEGF_TRY(mm(true, b(sl), b(a), P0, prow, spr, P0, Vp(a), (int64_t)b(a) * P0, b(a), s.Gb(sl, a), sG, b(a), -1.0, true));
        }
      }
    // separator band blocks (right separator of this domain): G_S itself
    const int s0 = l + 1;
    for (int a = s0; a < s0 + w; ++a)
      for (int c = s0; c < s0 + w; ++c)
        NEGF_TRY(cp(GSd(j) + (int64_t)p->off_in[a] * P + p->off_in[c], sPP, P, s.Gb(a, c), sG, b(c), b(a), b(c), 1.0, 0, C));
    return cudaSuccess;
  }

  // G_1N = G_{1,N}: layer 1 is in D2_1 and layer N in the last separator:
  // G_{1,N} = -W_1 (T_S^{-1})_{p_1, p_n}[:, N].
  cudaError_t g1n(double2* out, int64_t sOut) {
    const int N = p->N, P0 = p->Psz[0], Pn = p->Psz[nd - 1];
    return mm(true, b(0), b(N - 1), P0, Wq(0), (int64_t)b(0) * P0, P0, RS(nd - 1) + p->off_in[N - 1],
              (int64_t)P0 * Pn, Pn, out, sOut, b(N - 1), -1.0, false);
  }

  // Runs f(dd_j, j) for every sub-domain j concurrently: domain j of this
  // energy group on its own stream (graph branch), joined back afterwards.
  // Each domain sweeps in its own Schur-window slots; everything else a
  // domain writes (its layers' halos, W / V / Z, band blocks next to its
  // separators) is disjoint from the other domains'.
  template <class F>
  cudaError_t for_domains(F f) {
    const int g = s.grp;
    NEGF_TRY(cudaEventRecord(p->dfork[g], s.st));
    for (int j = 1; j < nd; ++j) NEGF_TRY(cudaStreamWaitEvent(p->dstream[(size_t)g * nd + j], p->dfork[g], 0));
    for (int j = 0; j < nd; ++j) {
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
    for (int j = 1; j < nd; ++j) {
      NEGF_TRY(cudaEventRecord(p->djoin[(size_t)g * nd + j], p->dstream[(size_t)g * nd + j]));
      NEGF_TRY(cudaStreamWaitEvent(s.st, p->djoin[(size_t)g * nd + j], 0));
    }
    return cudaSuccess;
  }

  cudaError_t run(bool want_band, double2* g1n_out, int64_t s1) {
    NEGF_TRY(for_domains([&](DD& d, int j) { return d.domain(j); }));
    NEGF_TRY(schur());
    NEGF_TRY(interface(g1n_out != nullptr));
    if (want_band) NEGF_TRY(for_domains([&](DD& d, int j) { return d.stitch(j); }));
    if (g1n_out) NEGF_TRY(g1n(g1n_out, s1));
    return cudaSuccess;
  }
};

}  // namespace
