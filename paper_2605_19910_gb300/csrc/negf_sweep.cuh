// The RGF schedule of one call over one energy range (one TU: included by
// negf_capi.cu only): the upward and downward sweeps of Alg. 1 / Sec. 2.3,
// the G_1N chain, the last block column, refinement, transmission, the
// adjoint's pieces (also checkpointed) and the Keldysh recursion, each step
// a batched launch over the range's energies.
#pragma once

#include <algorithm>
#include <map>

#include "negf_plan.cuh"

namespace {

// ---------------------------------------------------------------------------
// One call's schedule.
// ---------------------------------------------------------------------------
struct Sweep {
  negf_plan_s* p;
  cudaStream_t st;
  const double2* H;
  const double2* sigL;
  const double2* sigR;
  int64_t sig_stride;
  const double2* E;
  double2* Gband;     // may be null
  double2* G1N;       // may be null
  int32_t* info;
  int e0, ne;         // energy range of this sweep
  int wofs = 0;       // energy offset of this range inside the chunk workspace
  int gb_e0 = 0;      // energy index of Gband[0] (0: caller's buffer; chunk start: internal buffer)
  int grp = 0;        // energy group (stream set) of this sweep
  int sdom = 0;       // DDRGF sub-domain: selects its own Schur-window slots
  cudaEvent_t after_first_inv = nullptr;   // recorded once, after this sweep's first inversion
  // Boundary self-energies of a DDRGF sub-domain solved as an open system:
  // xr (Sigma_right, rows / columns of layers xr_f .. xr_f + w - 1, leading
  // dimension xr_ld, per-energy stride xr_s) and xl (Sigma_left, layers
  // xl_f .. xl_f + w - 1) are subtracted from the Schur-window blocks of
  // those layers when upward() first forms them.
  const double2* xr = nullptr; int xr_f = -1, xr_ld = 0; int64_t xr_s = 0;
  const double2* xl = nullptr; int xl_f = -1, xl_ld = 0; int64_t xl_s = 0;
  // Host copy of the band (negf_solve_host with page-locked outputs): the
  // energy-major host band, the group's copy stream and event, the number of
  // layer pieces and the last layer already copied.
  double2* host_band = nullptr;
  cudaStream_t cst = nullptr;
  cudaEvent_t cready = nullptr;
  int host_pieces = 4, host_done = -1;

  // Copy to the host every band block (a, b) with max(a, b) <= i not copied
  // yet: for each diagonal d a contiguous run of blocks per energy, one 2-D
  // copy over the range's energies (pitch: one band), on the copy stream
  // after this stream's work so far.
  cudaError_t host_copy_upto(int i) {
    const int N = p->N, w = p->w;
    NEGF_TRY(cudaEventRecord(cready, st));
    NEGF_TRY(cudaStreamWaitEvent(cst, cready, 0));
    const size_t pitch = (size_t)p->band_elems * sizeof(double2);
    for (int d = -w; d <= w; ++d) {
      const int lo = std::max(std::max(0, -d), host_done - std::max(0, d) + 1);
      const int hi = std::min(std::min(N - 1, N - 1 - d), i - std::max(0, d));
      if (hi < lo) continue;
      const int64_t o0 = p->band_off[(size_t)(d + w) * N + lo];
      const int64_t o1 = p->band_off[(size_t)(d + w) * N + hi] + (int64_t)p->b[hi] * p->b[hi + d];
      const size_t width = (size_t)(o1 - o0) * sizeof(double2);
      NEGF_TRY(cudaMemcpy2DAsync(host_band + (int64_t)e0 * p->band_elems + o0, pitch,
                                 Gband + (int64_t)(e0 - gb_e0) * p->band_elems + o0, pitch, width, (size_t)ne,
                                 cudaMemcpyDeviceToHost, cst));
    }
    host_done = i;
    return cudaSuccess;
  }
  // After layer i of a downward pass over [f, l]: copy at piece boundaries.
  cudaError_t host_copy_after(int i, int f, int l) {
    if (!host_band) return cudaSuccess;
    const int n = l - f + 1, k = i - f + 1;
    const bool boundary = i == l || (k * host_pieces) / n != ((k - 1) * host_pieces) / n;
    return boundary ? host_copy_upto(i) : cudaSuccess;
  }

  // Offset of layer a inside the w layers starting at layer a0.
  int off_from(int a0, int a) const {
    int o = 0;
    for (int k = a0; k < a; ++k) o += p->b[k];
    return o;
  }
  // The boundary block subtracted from S_ab (nullptr if none).
  const double2* boundary(int a, int bb, int64_t* stride, int* ld) const {
    const int w = p->w;
    if (xr && a >= xr_f && a < xr_f + w && bb >= xr_f && bb < xr_f + w) {
      *stride = xr_s; *ld = xr_ld;
      return xr + (int64_t)off_from(xr_f, a) * xr_ld + off_from(xr_f, bb);
    }
    if (xl && a >= xl_f && a < xl_f + w && bb >= xl_f && bb < xl_f + w) {
      *stride = xl_s; *ld = xl_ld;
      return xl + (int64_t)off_from(xl_f, a) * xl_ld + off_from(xl_f, bb);
    }
    return nullptr;
  }

  // Every kernel launch of the schedule goes through here so that the
  // optional profiler can bracket it with events on the launching stream.
  template <class F>
  cudaError_t launch(int kind, double flops, F f) { return launch(kind, flops, flops, f); }
  template <class F>
  cudaError_t launch(int kind, double flops, double issued, F f) {
    if (!p->profiling) return f();
    negf_plan_s::Rec r{kind, flops, issued, nullptr, nullptr};
    NEGF_TRY(cudaEventCreate(&r.a));
    NEGF_TRY(cudaEventCreate(&r.b));
    NEGF_TRY(cudaEventRecord(r.a, st));
    cudaError_t e = f();
    NEGF_TRY(cudaEventRecord(r.b, st));
    p->recs.push_back(r);
    return e;
  }
  static double gemm_flops(const ZGemm& g) {
    return 8.0 * g.m * (double)g.n * g.k * g.batch;
  }
  cudaError_t gemm(ZGemm g) {
    g.errword = p->d_err;
    g.wait_limit = p->wait_limit;
    g.tc_cols = p->tc_cols;
    if (g.bits == 0) g.bits = p->bits;
    if (p->precision == NEGF_MIXED)
      return launch(NEGF_PROF_GEMM_TC, gemm_flops(g), p->profiling ? negf::zgemm_tc_issued_flops(g) : 0.0,
                    [&] { return negf::zgemm_tc(g, st); });
    return gemm64(g);
  }
  cudaError_t gemm64(ZGemm g) {
    return launch(NEGF_PROF_GEMM_F64, gemm_flops(g), p->profiling ? negf::zgemm_f64_issued_flops(g) : 0.0,
                  [&] { return negf::zgemm_f64(g, st); });
  }
  cudaError_t inv(const double2* S, int64_t sS, double2* T, int64_t sT, int b, int batch, int layer1) {
    NEGF_TRY(launch(NEGF_PROF_INV, 8.0 * b * (double)b * b * batch, [&] {
      return negf::zinv_f64(S, sS, T, sT, b, batch, info + e0, layer1, p->d_err, st);
    }));
    if (after_first_inv) {
      NEGF_TRY(cudaEventRecord(after_first_inv, st));
      after_first_inv = nullptr;
    }
    return cudaSuccess;
  }
  template <class F>
  cudaError_t misc(F f) { return launch(NEGF_PROF_MISC, 0.0, f); }
  const double2* Hblk(int a, int bb) const { return H + p->band_off[(bb - a + p->w) * p->N + a]; }
  double2* Tblk(int i) const { return p->T_ws + p->t_off[i] * p->chunk + (int64_t)wofs * sq(p->b[i]); }
  double2* Xblk(int i, int c) const {
    return p->X_ws + p->x_off[i * p->w + (i - c - 1)] * p->chunk + (int64_t)wofs * p->b[i] * p->b[c];
  }
  double2* Yblk(int c, int i) const {
    return p->Y_ws + p->y_off[i * p->w + (i - c - 1)] * p->chunk + (int64_t)wofs * p->b[c] * p->b[i];
  }
  double2* Sslot(int a, int bb) const {
    int r = p->w + 1;
    return p->S_ws + ((int64_t)sdom * r * r + (a % r) * r + (bb % r)) * p->s_slot * p->chunk + (int64_t)wofs * p->s_slot;
  }
  // Per-energy stride inside a shared slot is fixed (bmax^2, b_1 * bmax):
  // concurrent energy groups can be at different layers of different sizes.
  int64_t sS() const { return p->s_slot; }
  int64_t sR(int j) const { return p->full_row ? (int64_t)p->b[0] * p->b[j] : (int64_t)p->b[0] * p->r_elems; }
  double2* Gb(int a, int bb) const {
    return Gband + (int64_t)(e0 - gb_e0) * p->band_elems + p->band_off[(bb - a + p->w) * p->N + a];
  }
  // Lead self-energies of this energy range: Sigma_L acts on layer 0 and
  // Sigma_R on layer N-1 (the same layer when N == 1).
  const double2* sigmaL() const { return sigL ? sigL + (sig_stride ? (int64_t)e0 * sig_stride : 0) : nullptr; }
  const double2* sigmaR() const { return sigR ? sigR + (sig_stride ? (int64_t)e0 * sig_stride : 0) : nullptr; }

  // Upward pass (Alg. 1 upward loop / Sec. 2.3): eliminate layers l .. f of
  // the chain restricted to [f, l] (the whole chain by default; one DDRGF
  // sub-domain otherwise).  Sigma_L / Sigma_R enter only if layer 0 / N-1 is
  // inside the range.
  cudaError_t upward(bool need_x, int f = 0, int l = -1) {
    const int N = p->N, w = p->w, C = ne;
    if (l < 0) l = N - 1;
    std::map<std::pair<int, int>, bool> mat;   // S_ab materialized per energy
    // S_{l,l} = E I - H_ll (- Sigma_R if l = N-1) (- Sigma_L if l = 0)
    {
      int bl = p->b[l];
      double2* dst = Sslot(l, l);
      const double2* extra = (l == N - 1) ? sigmaR() : nullptr;
      NEGF_TRY(misc([&] {
        return negf::assemble_diag(Hblk(l, l), E + e0, extra, sig_stride, dst, sS(), bl, C, st);
      }));
      if (l == 0 && sigL) {
        ZGemm g;   // dst -= Sigma_L : expressed as C = 1*dst - 1*SigmaL with an empty product
        g.m = bl; g.n = bl; g.k = 0;
        g.A = dst; g.B = dst; g.lda = bl; g.ldb = bl;
        g.C = dst; g.sC = sS(); g.ldc = bl;
        g.C1 = dst; g.sC1 = sS(); g.ldc1 = bl; g.beta1 = {1.0, 0.0};
        g.C2 = sigmaL(); g.sC2 = sig_stride; g.ldc2 = bl; g.beta2 = {-1.0, 0.0};
        g.batch = C;
        NEGF_TRY(gemm64(g));
      }
      mat[{l, l}] = true;
    }
    if (xr) {
      // the trailing window [xr_f, l] carries Sigma_right from the start:
      // S_ab = E delta_ab I - H_ab - Sigma_right[a, b] for a, b in it
      for (int a = xr_f; a <= l; ++a)
        for (int bb = xr_f; bb <= l; ++bb) {
          int64_t bs = 0; int bld = 0;
          const double2* x = boundary(a, bb, &bs, &bld);
          const int ba = p->b[a], bbs = p->b[bb];
          double2* dst = Sslot(a, bb);
          if (a == l && bb == l) {
            NEGF_TRY(misc([&] { return negf::copy2d(x, bs, bld, dst, sS(), bbs, ba, bbs, -1.0, 1, C, st); }));
            continue;
          }
          ZGemm g;   // k = 0: C = -H_ab (+ E I) - Sigma_right[a, b]
          g.m = ba; g.n = bbs; g.k = 0;
          g.A = dst; g.B = dst; g.lda = bbs; g.ldb = bbs;
          g.C = dst; g.sC = sS(); g.ldc = bbs;
          g.C1 = Hblk(a, bb); g.sC1 = 0; g.ldc1 = bbs; g.beta1 = {-1.0, 0.0};
          g.C2 = x; g.sC2 = bs; g.ldc2 = bld; g.beta2 = {-1.0, 0.0};
          if (a == bb) { g.dshift = E + e0; g.sD = 1; g.gamma = {1.0, 0.0}; }
          g.batch = C;
          NEGF_TRY(gemm64(g));
          mat[{a, bb}] = true;
        }
    }
    for (int i = l; i >= f; --i) {
      const int bi = p->b[i];
      NEGF_TRY(inv(Sslot(i, i), sS(), Tblk(i), sq(bi), bi, C, i + 1));
      const int lo = std::max(f, i - w);
      for (int c = lo; c < i; ++c) {
        const int bc = p->b[c];
        const bool mic = mat.count({i, c}) > 0, mci = mat.count({c, i}) > 0;
        if (need_x) {   // X_{i,c} = t_i S_{i,c}
          ZGemm g;
          g.m = bi; g.n = bc; g.k = bi;
          g.A = Tblk(i); g.sA = sq(bi); g.lda = bi;
          if (mic) { g.B = Sslot(i, c); g.sB = sS(); g.ldb = bc; g.alpha = {1.0, 0.0}; }
          else { g.B = Hblk(i, c); g.sB = 0; g.ldb = bc; g.alpha = {-1.0, 0.0}; }
          g.C = Xblk(i, c); g.sC = (int64_t)bi * bc; g.ldc = bc;
          g.batch = C;
          NEGF_TRY(gemm(g));
        }
        {   // Y_{c,i} = S_{c,i} t_i
          ZGemm g;
          g.m = bc; g.n = bi; g.k = bi;
          if (mci) { g.A = Sslot(c, i); g.sA = sS(); g.lda = bi; g.alpha = {1.0, 0.0}; }
          else { g.A = Hblk(c, i); g.sA = 0; g.lda = bi; g.alpha = {-1.0, 0.0}; }
          g.B = Tblk(i); g.sB = sq(bi); g.ldb = bi;
          g.C = Yblk(c, i); g.sC = (int64_t)bc * bi; g.ldc = bi;
          g.batch = C;
          NEGF_TRY(gemm(g));
        }
      }
      // Window update S_ab -= Y_{a,i} S_{i,b}  (= S_{a,i} t_i S_{i,b}), a, b in [i-w, i-1]
      for (int a = lo; a < i; ++a) {
        for (int bb = lo; bb < i; ++bb) {
          const int ba = p->b[a], bbs = p->b[bb];
          const bool mib = mat.count({i, bb}) > 0, mab = mat.count({a, bb}) > 0;
          ZGemm g;
          g.m = ba; g.n = bbs; g.k = bi;
          g.A = Yblk(a, i); g.sA = (int64_t)ba * bi; g.lda = bi;
          if (mib) { g.B = Sslot(i, bb); g.sB = sS(); g.ldb = bbs; g.alpha = {-1.0, 0.0}; }
          else { g.B = Hblk(i, bb); g.sB = 0; g.ldb = bbs; g.alpha = {1.0, 0.0}; }
          double2* out = Sslot(a, bb);
          g.C = out; g.sC = sS(); g.ldc = bbs;
          if (mab) { g.C1 = out; g.sC1 = sS(); g.ldc1 = bbs; g.beta1 = {1.0, 0.0}; }
          else {
            g.C1 = Hblk(a, bb); g.sC1 = 0; g.ldc1 = bbs; g.beta1 = {-1.0, 0.0};
            if (a == bb) {
              g.dshift = E + e0; g.sD = 1; g.gamma = {1.0, 0.0};
              const double2* sg = nullptr;
              if (a == 0) sg = sigmaL();
              if (sg) { g.C2 = sg; g.sC2 = sig_stride; g.ldc2 = ba; g.beta2 = {-1.0, 0.0}; }
            }
            int64_t bs = 0; int bld = 0;
            const double2* x = boundary(a, bb, &bs, &bld);
            if (x) {   // a DDRGF sub-domain's Sigma_left (never on layer 0, which has no left neighbour)
              if (g.C2) return cudaErrorInvalidValue;
              g.C2 = x; g.sC2 = bs; g.ldc2 = bld; g.beta2 = {-1.0, 0.0};
            }
          }
          g.batch = C;
          NEGF_TRY(gemm(g));
          mat[{a, bb}] = true;
        }
      }
    }
    return cudaSuccess;
  }

  // Downward pass (Alg. 1 downward loop / Sec. 2.3) over [f, l], written into Gband.
  cudaError_t downward(int f = 0, int l = -1) {
    const int N = p->N, w = p->w, C = ne;
    if (l < 0) l = N - 1;
    const int64_t sG = p->band_elems;
    NEGF_TRY(misc([&] { return negf::copy_blocks(Tblk(f), sq(p->b[f]), Gb(f, f), sG, sq(p->b[f]), C, st); }));
    NEGF_TRY(host_copy_after(f, f, l));
    for (int i = f + 1; i <= l; ++i) {
      const int bi = p->b[i];
      const int lo = std::max(f, i - w);
      for (int a = lo; a < i; ++a) {     // G_{a,i} = -sum_c G_{a,c} Y_{c,i}
        for (int c = lo; c < i; ++c) {
          ZGemm g;
          g.m = p->b[a]; g.n = bi; g.k = p->b[c];
          g.A = Gb(a, c); g.sA = sG; g.lda = p->b[c];
          g.B = Yblk(c, i); g.sB = (int64_t)p->b[c] * bi; g.ldb = bi;
          g.C = Gb(a, i); g.sC = sG; g.ldc = bi; g.alpha = {-1.0, 0.0};
          if (c > lo) { g.C1 = Gb(a, i); g.sC1 = sG; g.ldc1 = bi; g.beta1 = {1.0, 0.0}; }
          g.batch = C;
          NEGF_TRY(gemm(g));
        }
      }
      for (int bb = lo; bb < i; ++bb) {  // G_{i,b} = -sum_c X_{i,c} G_{c,b}
        for (int c = lo; c < i; ++c) {
          ZGemm g;
          g.m = bi; g.n = p->b[bb]; g.k = p->b[c];
          g.A = Xblk(i, c); g.sA = (int64_t)bi * p->b[c]; g.lda = p->b[c];
          g.B = Gb(c, bb); g.sB = sG; g.ldb = p->b[bb];
          g.C = Gb(i, bb); g.sC = sG; g.ldc = p->b[bb]; g.alpha = {-1.0, 0.0};
          if (c > lo) { g.C1 = Gb(i, bb); g.sC1 = sG; g.ldc1 = p->b[bb]; g.beta1 = {1.0, 0.0}; }
          g.batch = C;
          NEGF_TRY(gemm(g));
        }
      }
      for (int c = lo; c < i; ++c) {     // G_ii = t_i - sum_c X_{i,c} G_{c,i}
        ZGemm g;
        g.m = bi; g.n = bi; g.k = p->b[c];
        g.A = Xblk(i, c); g.sA = (int64_t)bi * p->b[c]; g.lda = p->b[c];
        g.B = Gb(c, i); g.sB = sG; g.ldb = bi;
        g.C = Gb(i, i); g.sC = sG; g.ldc = bi; g.alpha = {-1.0, 0.0};
        if (c == lo) { g.C1 = Tblk(i); g.sC1 = sq(bi); g.ldc1 = bi; g.beta1 = {1.0, 0.0}; }
        else { g.C1 = Gb(i, i); g.sC1 = sG; g.ldc1 = bi; g.beta1 = {1.0, 0.0}; }
        g.batch = C;
        NEGF_TRY(gemm(g));
      }
      NEGF_TRY(host_copy_after(i, f, l));
    }
    return cudaSuccess;
  }

  // First block row G_{1,j} = -sum_c G_{1,c} Y_{c,j} (Eq. 4x4_exact_RGF, first
  // row); R_ws holds either the whole row (gradient) or a ring of w + 1.
  double2* Rblk(int j) const {
    const int64_t o = (int64_t)wofs * sR(j);
    if (p->full_row) return p->R_ws + p->r_off[j] * p->chunk + o;
    return p->R_ws + (int64_t)(j % (p->w + 1)) * (int64_t)p->b[0] * p->r_elems * p->chunk + o;
  }
  cudaError_t first_row(double2* g1n_out, int64_t s_out) {
    const int N = p->N, w = p->w, C = ne;
    const int b0 = p->b[0];
    if (N == 1) {
      if (p->full_row)
        NEGF_TRY(misc([&] { return negf::copy_blocks(Tblk(0), sq(b0), Rblk(0), sR(0), sq(b0), C, st); }));
      return misc([&] { return negf::copy_blocks(Tblk(0), sq(b0), g1n_out, s_out, sq(b0), C, st); });
    }
    NEGF_TRY(misc([&] { return negf::copy_blocks(Tblk(0), sq(b0), Rblk(0), sR(0), sq(b0), C, st); }));
    for (int j = 1; j < N; ++j) {
      const int bj = p->b[j];
      const int lo = std::max(0, j - w);
      const bool last = (j == N - 1);
      double2* out = last ? g1n_out : Rblk(j);
      const int64_t so = last ? s_out : sR(j);
      for (int c = lo; c < j; ++c) {
        ZGemm g;
        g.m = b0; g.n = bj; g.k = p->b[c];
        g.A = Rblk(c); g.sA = sR(c); g.lda = p->b[c];
        g.B = Yblk(c, j); g.sB = (int64_t)p->b[c] * bj; g.ldb = bj;
        g.C = out; g.sC = so; g.ldc = bj; g.alpha = {-1.0, 0.0};
        if (c > lo) { g.C1 = out; g.sC1 = so; g.ldc1 = bj; g.beta1 = {1.0, 0.0}; }
        g.batch = C;
        NEGF_TRY(gemm(g));
      }
      if (last && p->full_row)
        NEGF_TRY(misc([&] { return negf::copy_blocks(out, so, Rblk(j), sR(j), (int64_t)b0 * bj, C, st); }));
    }
    return cudaSuccess;
  }

  // Scratch slot k (0: Gamma_L, 1: Gamma_R, 2: P, 3: Q, 4: G_1N, 5, 6: gradient
  // temporaries) of this energy range; per-energy stride scr_stride(k).
  int64_t scr_stride(int k) const {
    const int b0 = p->b[0], bN = p->b[p->N - 1];
    return k == 0 ? sq(b0) : (k == 1 ? sq(bN) : (int64_t)b0 * bN);
  }
  double2* scr(int k) const {
    const int b0 = p->b[0], bN = p->b[p->N - 1];
    int64_t off = 0;
    for (int j = 0; j < k; ++j) off += (j == 0 ? sq(b0) : (j == 1 ? sq(bN) : (int64_t)b0 * bN)) * p->chunk;
    (void)b0; (void)bN;
    return p->scratch + off + (int64_t)wofs * scr_stride(k);
  }
  double2* Pblk(int i) const { return p->P_ws + p->p_off[i] * p->chunk + (int64_t)wofs * p->b[i] * p->b[p->N - 1]; }
  double2* LCblk(int i) const { return p->LC_ws + p->p_off[i] * p->chunk + (int64_t)wofs * p->b[i] * p->b[p->N - 1]; }

  // Last block column G_{i,N} (adjoint sweep).  With the factorisation
  // M = U D L of the upward pass (U_{i,i+1} = Y_{i,i+1}, L_{i+1,i} = X_{i+1,i},
  // D = diag(S_i); Eq. 2x2_UDL_factorization applied layer by layer), column N
  // of M^{-1} = L^{-1} D^{-1} U^{-1} e_N is:
  //   P_{N} = I,  P_i = -Y_{i,i+1} P_{i+1}            (U^{-1} e_N)
  //   G_{1,N}' = t_1 P_1,  G_{i,N} = t_i P_i - X_{i,i-1} G_{i-1,N}.
  cudaError_t last_column() {
    const int N = p->N, w = p->w, C = ne, bN = p->b[N - 1];
    for (int i = N - 1; i >= 0; --i) {   // P = U^{-1} e_N
      const int bi = p->b[i];
      if (i == N - 1) {
        NEGF_TRY(misc([&] { return negf::set_identity(Pblk(i), sq(bN), bN, C, st); }));
        continue;
      }
      for (int c = i + 1; c <= std::min(N - 1, i + w); ++c) {   // P_i = -sum_c Y_{i,c} P_c
        ZGemm g;
        g.m = bi; g.n = bN; g.k = p->b[c];
        g.A = Yblk(i, c); g.sA = (int64_t)bi * p->b[c]; g.lda = p->b[c];
        g.B = Pblk(c); g.sB = (int64_t)p->b[c] * bN; g.ldb = bN;
        g.C = Pblk(i); g.sC = (int64_t)bi * bN; g.ldc = bN; g.alpha = {-1.0, 0.0};
        if (c > i + 1) { g.C1 = Pblk(i); g.sC1 = (int64_t)bi * bN; g.ldc1 = bN; g.beta1 = {1.0, 0.0}; }
        g.batch = C;
        NEGF_TRY(gemm(g));
      }
    }
    for (int i = 0; i < N; ++i) {        // G_{i,N} = t_i P_i - sum_c X_{i,c} G_{c,N}
      const int bi = p->b[i];
      ZGemm g;
      g.m = bi; g.n = bN; g.k = bi;
      g.A = Tblk(i); g.sA = sq(bi); g.lda = bi;
      g.B = Pblk(i); g.sB = (int64_t)bi * bN; g.ldb = bN;
      g.C = LCblk(i); g.sC = (int64_t)bi * bN; g.ldc = bN;
      g.batch = C;
      NEGF_TRY(gemm(g));
      for (int c = std::max(0, i - w); c < i; ++c) {
        ZGemm h;
        h.m = bi; h.n = bN; h.k = p->b[c];
        h.A = Xblk(i, c); h.sA = (int64_t)bi * p->b[c]; h.lda = p->b[c];
        h.B = LCblk(c); h.sB = (int64_t)p->b[c] * bN; h.ldb = bN;
        h.C = LCblk(i); h.sC = (int64_t)bi * bN; h.ldc = bN; h.alpha = {-1.0, 0.0};
        h.C1 = LCblk(i); h.sC1 = (int64_t)bi * bN; h.ldc1 = bN; h.beta1 = {1.0, 0.0};
        h.batch = C;
        NEGF_TRY(gemm(h));
      }
    }
    return cudaSuccess;
  }

  // One step of iterative refinement of G_1N = x_1, x = M^{-1} e_N the last
  // block column (mixed precision; gives G_1N and T(E) to FP64-level
  // accuracy):
  //   r = e_N - M x with FP64-accurate products (56-bit tensor-core split,
  //       exact integer accumulation, the E x term in FP64),
  //   x_1 <- x_1 + (L^{-1} D^{-1} U^{-1} r)_1 = x_1 + t_1 (U^{-1} r)_1,
  // since L (L_{i,i-1} = X_{i,i-1}) is unit lower block triangular, so the
  // first block row of L^{-1} is e_1^T: only the backward pass v = U^{-1} r
  // and one product with t_1 are needed.  r / v live in the P region (free
  // after last_column); the refined G_1N goes to g1n_out.
  cudaError_t refine_g1n(double2* g1n_out, int64_t s_out) {
    const int N = p->N, w = p->w, C = ne, bN = p->b[N - 1];
    auto hx = [&](int i, int c, const double2* Aop, int64_t sA, int lda, double2* out, bool acc) {
      ZGemm g;   // out (+)= Aop * x_c, 56-bit products
      g.m = p->b[i]; g.n = bN; g.k = p->b[c];
      g.A = Aop; g.sA = sA; g.lda = lda;
      g.B = LCblk(c); g.sB = (int64_t)p->b[c] * bN; g.ldb = bN;
      g.C = out; g.sC = (int64_t)p->b[i] * bN; g.ldc = bN;
      if (acc) { g.C1 = out; g.sC1 = g.sC; g.ldc1 = bN; g.beta1 = {1.0, 0.0}; }
      g.bits = 56;
      g.batch = C;
      return gemm(g);
    };
    for (int i = 0; i < N; ++i) {   // r_i = delta_{i,N} I + sum_c H_{i,c} x_c - E x_i + Sigma_i x_i
      const int bi = p->b[i];
      bool acc = false;
      for (int c = std::max(0, i - w); c <= std::min(N - 1, i + w); ++c) {
        NEGF_TRY(hx(i, c, Hblk(i, c), 0, p->b[c], Pblk(i), acc));
        acc = true;
      }
      if (i == 0 && sigL) NEGF_TRY(hx(0, 0, sigmaL(), sig_stride, bi, Pblk(0), true));
      if (i == N - 1 && sigR) NEGF_TRY(hx(i, i, sigmaR(), sig_stride, bi, Pblk(i), true));
      NEGF_TRY(misc([&] {
        return negf::axpy_scalar(Pblk(i), (int64_t)bi * bN, LCblk(i), (int64_t)bi * bN, E + e0, -1.0, bi, bN, bN, C, st);
      }));
      if (i == N - 1)
        NEGF_TRY(misc([&] { return negf::add_diag(Pblk(i), sq(bN), bN, bN, nullptr, 0, 1.0, C, st); }));
    }
    for (int i = N - 2; i >= 0; --i)   // v = U^{-1} r (in place)
      for (int c = i + 1; c <= std::min(N - 1, i + w); ++c) {
        ZGemm g;
        g.m = p->b[i]; g.n = bN; g.k = p->b[c];
        g.A = Yblk(i, c); g.sA = (int64_t)p->b[i] * p->b[c]; g.lda = p->b[c];
        g.B = Pblk(c); g.sB = (int64_t)p->b[c] * bN; g.ldb = bN;
        g.C = Pblk(i); g.sC = (int64_t)p->b[i] * bN; g.ldc = bN; g.alpha = {-1.0, 0.0};
        g.C1 = Pblk(i); g.sC1 = g.sC; g.ldc1 = bN; g.beta1 = {1.0, 0.0};
        g.batch = C;
        NEGF_TRY(gemm(g));
      }
    const int b0 = p->b[0];
    ZGemm g;   // G_1N = x_1 + t_1 v_1
    g.m = b0; g.n = bN; g.k = b0;
    g.A = Tblk(0); g.sA = sq(b0); g.lda = b0;
    g.B = Pblk(0); g.sB = (int64_t)b0 * bN; g.ldb = bN;
    g.C = g1n_out; g.sC = s_out; g.ldc = bN;
    g.C1 = LCblk(0); g.sC1 = (int64_t)b0 * bN; g.ldc1 = bN; g.beta1 = {1.0, 0.0};
    g.batch = C;
    return gemm(g);
  }

  // K = Gamma_R G_1N^H Gamma_L (bN x b1) and U_a = K G_{1,a} (bN x b_a) for
  // every layer a, written over P (no longer needed).
  cudaError_t grad_prep(const double2* g1n, int64_t sG) {
    const int N = p->N, C = ne, b0 = p->b[0], bN = p->b[N - 1];
    NEGF_TRY(grad_K(g1n, sG));
    double2* K = scr(6);
    for (int a = 0; a < N; ++a) {   // U_a = K G_{1,a}
      const int ba = p->b[a];
      ZGemm g;
      g.m = bN; g.n = ba; g.k = b0;
      g.A = K; g.sA = (int64_t)bN * b0; g.lda = b0;
      g.B = Rblk(a); g.sB = sR(a); g.ldb = ba;
      g.C = Pblk(a); g.sC = (int64_t)ba * bN; g.ldc = ba;
      g.batch = C;
      NEGF_TRY(gemm(g));
    }
    return cudaSuccess;
  }

  // Gamma_L, Gamma_R (scratch 0, 1) and K = Gamma_R G_1N^H Gamma_L (scratch 6).
  cudaError_t grad_K(const double2* g1n, int64_t sG) {
    const int N = p->N, C = ne, b0 = p->b[0], bN = p->b[N - 1];
    const int nsig = sig_stride ? C : 1;
    double2* gL = scr(0);
    double2* gR = scr(1);
    double2* W = scr(5);
    double2* K = scr(6);
    NEGF_TRY(misc([&] { return negf::gamma_from_sigma(sigmaL(), sig_stride, gL, sq(b0), b0, nsig, st); }));
    NEGF_TRY(misc([&] { return negf::gamma_from_sigma(sigmaR(), sig_stride, gR, sq(bN), bN, nsig, st); }));
    {   // W = G_1N^H Gamma_L  (bN x b0)
      ZGemm g;
      g.m = bN; g.n = b0; g.k = b0;
      g.A = g1n; g.sA = sG; g.lda = bN; g.opA = negf::OP_C;
      g.B = gL; g.sB = sig_stride ? sq(b0) : 0; g.ldb = b0;
      g.C = W; g.sC = (int64_t)bN * b0; g.ldc = b0;
      g.batch = C;
      NEGF_TRY(gemm64(g));
    }
    {   // K = Gamma_R W
      ZGemm g;
      g.m = bN; g.n = b0; g.k = bN;
      g.A = gR; g.sA = sig_stride ? sq(bN) : 0; g.lda = bN;
      g.B = W; g.sB = (int64_t)bN * b0; g.ldb = b0;
      g.C = K; g.sC = (int64_t)bN * b0; g.ldc = b0;
      g.batch = C;
      NEGF_TRY(gemm64(g));
    }
    return cudaSuccess;
  }

  // ---- Keldysh equation G^< = G^R Sigma^< G^A (block tridiagonal) --------
  // Recursion over the factorisation M = U D L of the upward sweep (the
  // retarded band, t_i and X_{i,i-1} must be in place):
  //   upward   Q_i = Sigma^<_i + H_{i,i+1} g^<_{i+1} H_{i,i+1}^H,
  //            W_i = Q_i t_i^H,  g^<_i = t_i W_i;
  //   downward G^<_11 = g^<_1;  A_i = G^R_{i-1,i} W_i,
  //            G^<_{i,i-1} = -X_{i,i-1} G^<_{i-1,i-1} - A_i^H,
  //            G^<_{i-1,i} = -(G^<_{i,i-1})^H,
  //            G^<_ii = g^<_i - X_{i,i-1} A_i - G^<_{i,i-1} X_{i,i-1}^H.
  // Sigma^<_i: the leads' blocks on layers 1 and N plus an optional
  // per-energy scalar times I on every layer.  Products in the plan's
  // precision (the tensor-core kernel takes B^H operands).
  double2* LWblk(int i) const { return p->LW_ws + p->t_off[i] * p->chunk + (int64_t)wofs * sq(p->b[i]); }
  double2* LGblk(int i) const { return p->LG_ws + p->t_off[i] * p->chunk + (int64_t)wofs * sq(p->b[i]); }
  double2* Lb(double2* base, int a, int bb) const {
    return base + (int64_t)(e0 - gb_e0) * p->band_elems + p->band_off[(bb - a + p->w) * p->N + a];
  }
  cudaError_t lesser_up(const double2* slL, const double2* slR, int64_t sls, const double2* ldiag) {
    const int N = p->N, C = ne;
    double2* Q = Sslot(0, 0);
    double2* T1 = Sslot(0, 1);
    const double2* sLe = slL ? slL + (sls ? (int64_t)e0 * sls : 0) : nullptr;
    const double2* sRe = slR ? slR + (sls ? (int64_t)e0 * sls : 0) : nullptr;
    for (int i = N - 1; i >= 0; --i) {
      const int bi = p->b[i];
      if (i == N - 1) {
        NEGF_TRY(misc([&] { return negf::set_eye(Q, sS(), bi, bi, bi, 0, 0, 0, C, st); }));
      } else {
        const int bn = p->b[i + 1];
        ZGemm g;   // T1 = H_{i,i+1} g^<_{i+1}
        g.m = bi; g.n = bn; g.k = bn;
        g.A = Hblk(i, i + 1); g.sA = 0; g.lda = bn;
        g.B = LGblk(i + 1); g.sB = sq(bn); g.ldb = bn;
        g.C = T1; g.sC = sS(); g.ldc = bn;
        g.batch = C;
        NEGF_TRY(gemm(g));
        ZGemm h;   // Q = T1 H_{i,i+1}^H
        h.m = bi; h.n = bi; h.k = bn;
        h.A = T1; h.sA = sS(); h.lda = bn;
        h.B = Hblk(i, i + 1); h.sB = 0; h.ldb = bn; h.opB = negf::OP_C;
        h.C = Q; h.sC = sS(); h.ldc = bi;
        h.batch = C;
        NEGF_TRY(gemm(h));
      }
      if (i == 0 && sLe) NEGF_TRY(misc([&] { return negf::copy2d(sLe, sls, bi, Q, sS(), bi, bi, bi, 1.0, 1, C, st); }));
      if (i == N - 1 && sRe) NEGF_TRY(misc([&] { return negf::copy2d(sRe, sls, bi, Q, sS(), bi, bi, bi, 1.0, 1, C, st); }));
      if (ldiag) NEGF_TRY(misc([&] { return negf::add_diag(Q, sS(), bi, bi, ldiag + e0, 1, 1.0, C, st); }));
      ZGemm g;   // W_i = Q t_i^H
      g.m = bi; g.n = bi; g.k = bi;
      g.A = Q; g.sA = sS(); g.lda = bi;
      g.B = Tblk(i); g.sB = sq(bi); g.ldb = bi; g.opB = negf::OP_C;
      g.C = LWblk(i); g.sC = sq(bi); g.ldc = bi;
      g.batch = C;
      NEGF_TRY(gemm(g));
      ZGemm h;   // g^<_i = t_i W_i
      h.m = bi; h.n = bi; h.k = bi;
      h.A = Tblk(i); h.sA = sq(bi); h.lda = bi;
      h.B = LWblk(i); h.sB = sq(bi); h.ldb = bi;
      h.C = LGblk(i); h.sC = sq(bi); h.ldc = bi;
      h.batch = C;
      NEGF_TRY(gemm(h));
    }
    return cudaSuccess;
  }
  cudaError_t lesser_down(double2* Gl) {
    const int N = p->N, C = ne;
    const int64_t sG = p->band_elems;
    double2* Am = Sslot(0, 1);
    NEGF_TRY(misc([&] { return negf::copy_blocks(LGblk(0), sq(p->b[0]), Lb(Gl, 0, 0), sG, sq(p->b[0]), C, st); }));
    for (int i = 1; i < N; ++i) {
      const int bi = p->b[i], bc = p->b[i - 1];
      {
        ZGemm g;   // A_i = G^R_{i-1,i} W_i
        g.m = bc; g.n = bi; g.k = bi;
        g.A = Gb(i - 1, i); g.sA = sG; g.lda = bi;
        g.B = LWblk(i); g.sB = sq(bi); g.ldb = bi;
        g.C = Am; g.sC = sS(); g.ldc = bi;
        g.batch = C;
        NEGF_TRY(gemm(g));
      }
      double2* low = Lb(Gl, i, i - 1);
      {
        ZGemm g;   // G^<_{i,i-1} = -X_{i,i-1} G^<_{i-1,i-1} ...
        g.m = bi; g.n = bc; g.k = bc;
        g.A = Xblk(i, i - 1); g.sA = (int64_t)bi * bc; g.lda = bc;
        g.B = Lb(Gl, i - 1, i - 1); g.sB = sG; g.ldb = bc;
        g.C = low; g.sC = sG; g.ldc = bc; g.alpha = {-1.0, 0.0};
        g.batch = C;
        NEGF_TRY(gemm(g));
      }
      // ... - A_i^H; then G^<_{i-1,i} = -(G^<_{i,i-1})^H
      NEGF_TRY(misc([&] { return negf::copy2d_ct(Am, sS(), bi, low, sG, bc, bi, bc, -1.0, 1, C, st); }));
      NEGF_TRY(misc([&] { return negf::copy2d_ct(low, sG, bc, Lb(Gl, i - 1, i), sG, bi, bc, bi, -1.0, 0, C, st); }));
      double2* dia = Lb(Gl, i, i);
      {
        ZGemm g;   // G^<_ii = g^<_i - X_{i,i-1} A_i ...
        g.m = bi; g.n = bi; g.k = bc;
        g.A = Xblk(i, i - 1); g.sA = (int64_t)bi * bc; g.lda = bc;
        g.B = Am; g.sB = sS(); g.ldb = bi;
        g.C = dia; g.sC = sG; g.ldc = bi; g.alpha = {-1.0, 0.0};
        g.C1 = LGblk(i); g.sC1 = sq(bi); g.ldc1 = bi; g.beta1 = {1.0, 0.0};
        g.batch = C;
        NEGF_TRY(gemm(g));
      }
      {
        ZGemm g;   // ... - G^<_{i,i-1} X_{i,i-1}^H
        g.m = bi; g.n = bi; g.k = bc;
        g.A = low; g.sA = sG; g.lda = bc;
        g.B = Xblk(i, i - 1); g.sB = (int64_t)bi * bc; g.ldb = bc; g.opB = negf::OP_C;
        g.C = dia; g.sC = sG; g.ldc = bi; g.alpha = {-1.0, 0.0};
        g.C1 = dia; g.sC1 = sG; g.ldc1 = bi; g.beta1 = {1.0, 0.0};
        g.batch = C;
        NEGF_TRY(gemm(g));
      }
    }
    return cudaSuccess;
  }

  // ---- checkpointed adjoint (block tridiagonal) ----------------------------
  // Rings of k + 1 layers with fixed per-energy strides (bmax^2 for t, X, Y;
  // bmax * b_N for P / U and the last column); X_{i,i-1} and Y_{i-1,i} sit in
  // the slot of layer i.  Segment sg covers layers [sg k, min(N, (sg+1) k) - 1].
  int ck_slot(int i) const { return i % (p->ck_k + 1); }
  double2* ck_ring(double2* base, int i, int64_t stride) const {
    return base + (int64_t)ck_slot(i) * stride * p->chunk + (int64_t)wofs * stride;
  }
  double2* cT(int i) const { return ck_ring(p->T_ws, i, p->bmax2); }
  double2* cX(int i) const { return ck_ring(p->X_ws, i, p->bmax2); }
  double2* cY(int i) const { return ck_ring(p->Y_ws, i, p->bmax2); }
  double2* cP(int i) const { return ck_ring(p->P_ws, i, p->bmaxN); }
  double2* cL(int i) const { return ck_ring(p->LC_ws, i, p->bmaxN); }
  double2* ckS(int sg) const { return p->CKS + (int64_t)sg * p->bmax2 * p->chunk + (int64_t)wofs * p->bmax2; }
  double2* ckP(int sg) const { return p->CKP + (int64_t)sg * p->bmaxN * p->chunk + (int64_t)wofs * p->bmaxN; }
  int seg_lo(int sg) const { return sg * p->ck_k; }
  int seg_hi(int sg) const { return std::min(p->N, (sg + 1) * p->ck_k) - 1; }

  // Eliminate layer i: t_i = S_i^{-1}; for i > 0 the multipliers
  // X_{i,i-1} = t_i M_{i,i-1} (if want_x) and Y_{i-1,i} = M_{i-1,i} t_i; if
  // want_next also S_{i-1} = M_{i-1,i-1} - Y_{i-1,i} M_{i,i-1} and the suffix
  // product P_{i-1} = -Y_{i-1,i} P_i of U^{-1} e_N.
  cudaError_t ck_eliminate(int i, bool want_x, bool want_next) {
    const int C = ne, bi = p->b[i], bN = p->b[p->N - 1];
    const int64_t s2 = p->bmax2, sN = p->bmaxN;
    NEGF_TRY(inv(Sslot(i, i), sS(), cT(i), s2, bi, C, i + 1));
    if (i == 0) return cudaSuccess;
    const int bc = p->b[i - 1];
    if (want_x) {   // X_{i,i-1} = -t_i H_{i,i-1}
      ZGemm g;
      g.m = bi; g.n = bc; g.k = bi;
      g.A = cT(i); g.sA = s2; g.lda = bi;
      g.B = Hblk(i, i - 1); g.sB = 0; g.ldb = bc; g.alpha = {-1.0, 0.0};
      g.C = cX(i); g.sC = s2; g.ldc = bc;
      g.batch = C;
      NEGF_TRY(gemm(g));
    }
    {   // Y_{i-1,i} = -H_{i-1,i} t_i
      ZGemm g;
      g.m = bc; g.n = bi; g.k = bi;
      g.A = Hblk(i - 1, i); g.sA = 0; g.lda = bi; g.alpha = {-1.0, 0.0};
      g.B = cT(i); g.sB = s2; g.ldb = bi;
      g.C = cY(i); g.sC = s2; g.ldc = bi;
      g.batch = C;
      NEGF_TRY(gemm(g));
    }
    if (!want_next) return cudaSuccess;
    {   // S_{i-1} = E I - H_{i-1,i-1} (- Sigma_L on layer 0) + Y_{i-1,i} H_{i,i-1}
      ZGemm g;
      g.m = bc; g.n = bc; g.k = bi;
      g.A = cY(i); g.sA = s2; g.lda = bi;
      g.B = Hblk(i, i - 1); g.sB = 0; g.ldb = bc; g.alpha = {1.0, 0.0};
      double2* out = Sslot(i - 1, i - 1);
      g.C = out; g.sC = sS(); g.ldc = bc;
      g.C1 = Hblk(i - 1, i - 1); g.sC1 = 0; g.ldc1 = bc; g.beta1 = {-1.0, 0.0};
      g.dshift = E + e0; g.sD = 1; g.gamma = {1.0, 0.0};
      if (i - 1 == 0 && sigL) { g.C2 = sigmaL(); g.sC2 = sig_stride; g.ldc2 = bc; g.beta2 = {-1.0, 0.0}; }
      g.batch = C;
      NEGF_TRY(gemm(g));
    }
    {   // P_{i-1} = -Y_{i-1,i} P_i
      ZGemm g;
      g.m = bc; g.n = bN; g.k = bi;
      g.A = cY(i); g.sA = s2; g.lda = bi;
      g.B = cP(i); g.sB = sN; g.ldb = bN; g.alpha = {-1.0, 0.0};
      g.C = cP(i - 1); g.sC = sN; g.ldc = bN;
      g.batch = C;
      NEGF_TRY(gemm(g));
    }
    return cudaSuccess;
  }

  // Forward pass: the whole upward sweep with P_{N-1} = I and the suffix
  // products alongside, a checkpoint (S_hi, P_hi) before the top layer of
  // every segment but the first (the first stays in the rings), and
  // G_1N = t_1 P_1 (first block of the last column) at the end.
  cudaError_t ck_forward(double2* g1n_out, int64_t s_out) {
    const int N = p->N, C = ne, b0 = p->b[0], bN = p->b[N - 1], bl = p->b[N - 1];
    {   // S_{N-1} = E I - H - Sigma_R (- Sigma_L when N = 1)
      double2* dst = Sslot(N - 1, N - 1);
      NEGF_TRY(misc([&] {
        return negf::assemble_diag(Hblk(N - 1, N - 1), E + e0, sigmaR(), sig_stride, dst, sS(), bl, C, st);
      }));
      if (N == 1 && sigL) {
        ZGemm g;
        g.m = bl; g.n = bl; g.k = 0;
        g.A = dst; g.B = dst; g.lda = bl; g.ldb = bl;
        g.C = dst; g.sC = sS(); g.ldc = bl;
        g.C1 = dst; g.sC1 = sS(); g.ldc1 = bl; g.beta1 = {1.0, 0.0};
        g.C2 = sigmaL(); g.sC2 = sig_stride; g.ldc2 = bl; g.beta2 = {-1.0, 0.0};
        g.batch = C;
        NEGF_TRY(gemm64(g));
      }
    }
    NEGF_TRY(misc([&] { return negf::set_identity(cP(N - 1), p->bmaxN, bN, C, st); }));
    for (int i = N - 1; i >= 0; --i) {
      const int sg = i / p->ck_k, bi = p->b[i];
      if (sg >= 1 && i == seg_hi(sg)) {
        NEGF_TRY(misc([&] { return negf::copy_blocks(Sslot(i, i), sS(), ckS(sg), p->bmax2, sq(bi), C, st); }));
        NEGF_TRY(misc([&] {
          return negf::copy_blocks(cP(i), p->bmaxN, ckP(sg), p->bmaxN, (int64_t)bi * bN, C, st);
        }));
      }
      NEGF_TRY(ck_eliminate(i, sg == 0, true));
    }
    ZGemm g;   // G_1N = t_1 P_1
    g.m = b0; g.n = bN; g.k = b0;
    g.A = cT(0); g.sA = p->bmax2; g.lda = b0;
    g.B = cP(0); g.sB = p->bmaxN; g.ldb = bN;
    g.C = g1n_out; g.sC = s_out; g.ldc = bN;
    g.batch = C;
    return gemm(g);
  }

  // Recompute segment sg >= 1 from its checkpoint: layers hi .. lo, keeping
  // t, X, Y and P in the rings (the previous segment's top layer stays).
  cudaError_t ck_recompute(int sg) {
    const int C = ne, lo = seg_lo(sg), hi = seg_hi(sg), bh = p->b[hi], bN = p->b[p->N - 1];
    NEGF_TRY(misc([&] { return negf::copy_blocks(ckS(sg), p->bmax2, Sslot(hi, hi), sS(), sq(bh), C, st); }));
    NEGF_TRY(misc([&] { return negf::copy_blocks(ckP(sg), p->bmaxN, cP(hi), p->bmaxN, (int64_t)bh * bN, C, st); }));
    for (int i = hi; i >= lo; --i) NEGF_TRY(ck_eliminate(i, true, i > lo));
    return cudaSuccess;
  }

  // Reverse pass over segment sg, increasing layers: first row
  // G_{1,i} = -G_{1,i-1} Y_{i-1,i} (ring of two), last column
  // G_{i,N} = t_i P_i - X_{i,i-1} G_{i-1,N}, then U_i = K G_{1,i} over P_i.
  cudaError_t ck_chains(int sg) {
    const int C = ne, b0 = p->b[0], bN = p->b[p->N - 1];
    const int64_t s2 = p->bmax2, sN = p->bmaxN;
    double2* K = scr(6);
    for (int i = seg_lo(sg); i <= seg_hi(sg); ++i) {
      const int bi = p->b[i];
      if (i == 0) {
        NEGF_TRY(misc([&] { return negf::copy_blocks(cT(0), s2, Rblk(0), sR(0), sq(b0), C, st); }));
      } else {
        const int bc = p->b[i - 1];
        ZGemm g;
        g.m = b0; g.n = bi; g.k = bc;
        g.A = Rblk(i - 1); g.sA = sR(i - 1); g.lda = bc;
        g.B = cY(i); g.sB = s2; g.ldb = bi;
        g.C = Rblk(i); g.sC = sR(i); g.ldc = bi; g.alpha = {-1.0, 0.0};
        g.batch = C;
        NEGF_TRY(gemm(g));
      }
      {
        ZGemm g;   // G_{i,N} = t_i P_i
        g.m = bi; g.n = bN; g.k = bi;
        g.A = cT(i); g.sA = s2; g.lda = bi;
        g.B = cP(i); g.sB = sN; g.ldb = bN;
        g.C = cL(i); g.sC = sN; g.ldc = bN;
        g.batch = C;
        NEGF_TRY(gemm(g));
      }
      if (i > 0) {
        const int bc = p->b[i - 1];
        ZGemm h;   // G_{i,N} -= X_{i,i-1} G_{i-1,N}
        h.m = bi; h.n = bN; h.k = bc;
        h.A = cX(i); h.sA = s2; h.lda = bc;
        h.B = cL(i - 1); h.sB = sN; h.ldb = bN;
        h.C = cL(i); h.sC = sN; h.ldc = bN; h.alpha = {-1.0, 0.0};
        h.C1 = cL(i); h.sC1 = sN; h.ldc1 = bN; h.beta1 = {1.0, 0.0};
        h.batch = C;
        NEGF_TRY(gemm(h));
      }
      {
        ZGemm g;   // U_i = K G_{1,i}
        g.m = bN; g.n = bi; g.k = b0;
        g.A = K; g.sA = (int64_t)bN * b0; g.lda = b0;
        g.B = Rblk(i); g.sB = sR(i); g.ldb = bi;
        g.C = cP(i); g.sC = sN; g.ldc = bi;
        g.batch = C;
        NEGF_TRY(gemm(g));
      }
    }
    return cudaSuccess;
  }

  // T(E) = Re Tr[Gamma_L G_1N Gamma_R G_1N^H] from G_1N (stride sG).
  cudaError_t transmission(const double2* g1n, int64_t sG, double* T) {
    const int C = ne, b0 = p->b[0], bN = p->b[p->N - 1];
    double2* gL = p->scratch + (int64_t)wofs * sq(b0);
    double2* gR = p->scratch + sq(b0) * p->chunk + (int64_t)wofs * sq(bN);
    double2* Pm = p->scratch + (sq(b0) + sq(bN)) * p->chunk + (int64_t)wofs * b0 * bN;
    double2* Qm = p->scratch + (sq(b0) + sq(bN) + (int64_t)b0 * bN) * p->chunk + (int64_t)wofs * b0 * bN;
    const int nsig = sig_stride ? C : 1;
    NEGF_TRY(misc([&] { return negf::gamma_from_sigma(sigmaL(), sig_stride, gL, sq(b0), b0, nsig, st); }));
    NEGF_TRY(misc([&] { return negf::gamma_from_sigma(sigmaR(), sig_stride, gR, sq(bN), bN, nsig, st); }));
    {   // P = Gamma_L G_1N
      ZGemm g;
      g.m = b0; g.n = bN; g.k = b0;
      g.A = gL; g.sA = sig_stride ? sq(b0) : 0; g.lda = b0;
      g.B = g1n; g.sB = sG; g.ldb = bN;
      g.C = Pm; g.sC = (int64_t)b0 * bN; g.ldc = bN;
      g.batch = C;
      NEGF_TRY(gemm64(g));
    }
    {   // Q = Gamma_R G_1N^H
      ZGemm g;
      g.m = bN; g.n = b0; g.k = bN;
      g.A = gR; g.sA = sig_stride ? sq(bN) : 0; g.lda = bN;
      g.B = g1n; g.sB = sG; g.ldb = bN; g.opB = negf::OP_C;
      g.C = Qm; g.sC = (int64_t)bN * b0; g.ldc = b0;
      g.batch = C;
      NEGF_TRY(gemm64(g));
    }
    return misc([&] { return negf::trace_prod(Pm, (int64_t)b0 * bN, Qm, (int64_t)bN * b0, b0, bN, T + e0, C, 1.0, 0, st); });
  }
};

}  // namespace
