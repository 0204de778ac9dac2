// C-ABI of libnegf.so: plan construction, the schedule of the RGF sweep over
// a batch of energies, CUDA-graph capture of that schedule, and error folding.
//
// The sweep is Alg. 1 (block tridiagonal) generalised to a block n-diagonal
// matrix with half-bandwidth w (Sec. 2.3, Prop. 3 and the prose on the
// downward pass).  Every step runs for all energies of a chunk at once: each
// launch is one batched kernel over energies (the per-block inversion, or a
// block product whose H operand is shared by every energy).  The whole
// schedule of one call is captured once into a CUDA graph and replayed while
// the caller's pointers stay the same.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "../../include/negf.h"
#include "negf_common.cuh"
#include "negf_kernels.h"

using negf::ZGemm;

namespace {

struct BlockRef {        // where block S_ab of the running Schur complement lives
  bool materialized = false;
};

struct CallKey {
  const void* p[12];
  int64_t stride;
  int kind;
  bool operator==(const CallKey& o) const {
    return kind == o.kind && stride == o.stride && std::memcmp(p, o.p, sizeof(p)) == 0;
  }
};

}  // namespace

struct negf_plan_s {
  int N = 0, w = 1, nE = 0, n_domains = 1, precision = 0, refine = 0, outputs = 0, ckpt = 0, bits = 0;
  std::vector<int> b;
  std::vector<int64_t> band_off;   // (d + w) * N + i -> element offset or -1
  int64_t band_elems = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int chunk = 0;                   // energies per chunk

  // workspace (one allocation)
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int* d_err = nullptr;

  // per-energy element offsets inside one chunk slab of each region
  std::vector<int64_t> t_off, x_off, y_off;   // x_off/y_off indexed [i * w + (i - c - 1)]
  int64_t t_elems = 0, x_elems = 0, y_elems = 0;
  double2 *T_ws = nullptr, *X_ws = nullptr, *Y_ws = nullptr;
  double2* S_ws = nullptr;      // (w+1)^2 slots of bmax^2 per energy
  int64_t s_slot = 0;           // bmax^2
  double2* R_ws = nullptr;      // first-row chain: full row (grad) or a ring of w+1
  std::vector<int64_t> r_off;   // per layer offset (per energy) in R_ws
  int64_t r_elems = 0;
  double2* P_ws = nullptr;      // grad: suffix products P_i (b_i x b_N)
  double2* LC_ws = nullptr;     // grad: last column g_i (b_i x b_N)
  std::vector<int64_t> p_off;
  int64_t p_elems = 0;
  double2* RF_ws = nullptr;     // refinement: correction blocks (b_i x b_N)
  double2* scratch = nullptr;   // transmission: Gamma_L, Gamma_R, P, Q per energy
  int64_t scr_elems = 0;
  double2* G1N_ws = nullptr;    // G_1N when the caller does not keep it
  double* Tdummy = nullptr;
  bool full_row = false;        // R_ws holds the whole first row (adjoint without checkpoints)
  double2* DH_ws = nullptr;     // adjoint: per-energy products of one band pair (bmax^2 per energy)
  // negf_solve_host: device copies of the caller's host inputs / outputs
  // (allocated at the first call, sized for the sigma stride of that call)
  char* host_io = nullptr;
  size_t host_io_bytes = 0;
  double2* LW_ws = nullptr;     // Keldysh: W_i = Q_ii t_i^H per layer (t_i layout)
  double2* LG_ws = nullptr;     // Keldysh: right-connected g^<_i per layer

  // Checkpointed adjoint (checkpoint_every = k > 0): the sweep quantities
  // t_i, X_{i,i-1}, Y_{i-1,i}, P_i and the last column live in rings of k + 1
  // layers (fixed per-energy strides bmax^2 and bmax * b_N); the Schur
  // complement S_hi and P_hi at the top layer of every segment of k layers are
  // kept and the segment is recomputed from them in the reverse pass.
  int ck_k = 0, ck_nseg = 0;
  double2* CKS = nullptr;       // ck_nseg slots of bmax^2 per energy
  double2* CKP = nullptr;       // ck_nseg slots of bmax * b_N per energy
  int64_t bmax2 = 0, bmaxN = 0;

  // DDRGF (Alg. 2): n_domains (D2, D1) pairs; D2_j = [dom_f[j], dom_l[j]], its
  // right separator D1_j = [dom_l[j] + 1, dom_l[j] + w].
  std::vector<int> dom_f, dom_l, Fsz, Lsz, Psz;
  std::vector<int> dom_of;                       // layer -> domain (-1: separator)
  std::vector<int> sep_of;                       // layer -> separator (-1: domain)
  std::vector<int> off_in;                       // layer offset inside F / Lw / separator super-block
  std::vector<int64_t> fc_off, lc_off, wp_off, wq_off;   // per layer (D2 layers), per energy
  std::vector<int64_t> tsd_off, tsu_off, tsl_off, rs_off, ts_x_off;  // per separator
  std::vector<int64_t> mfp_off, mpf_off, mlq_off, mql_off;  // per domain, energy independent
  int64_t fc_e = 0, lc_e = 0, wp_e = 0, wq_e = 0, tsd_e = 0, tsu_e = 0, rs_e = 0, ts_x_e = 0, msup_e = 0;
  int Pmax = 0;
  double2 *FC = nullptr, *FR = nullptr, *LCd = nullptr, *LR = nullptr, *VT = nullptr;
  double2 *Wp = nullptr, *Wq = nullptr, *Vp = nullptr, *Vq = nullptr, *Zp = nullptr, *Zq = nullptr;
  double2 *TSd = nullptr, *TSu = nullptr, *TSl = nullptr, *GSd = nullptr, *GSu = nullptr, *GSl = nullptr;
  double2 *tS = nullptr, *XS = nullptr, *YS = nullptr, *SS = nullptr, *RS = nullptr, *Msup = nullptr;
  double2* band_ws = nullptr;   // band of one chunk when the caller keeps no band output

  // independent energy groups run on forked streams (graph branches)
  int groups = 1;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;   // [0] fork, [1..] joins
  std::vector<cudaEvent_t> stagger;   // group g -> g + 1 start dependency
  // DDRGF: the sub-domains of one energy group run concurrently, domain j of
  // group g on dstream[g * n_domains + j] (j = 0 on the group's own stream)
  std::vector<cudaStream_t> dstream;
  std::vector<cudaEvent_t> dfork, djoin;

  // optional per-launch timing (negf_profile_enable)
  bool profiling = false;
  struct Rec { int kind; double flops; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  double prof_ms[NEGF_PROF_KINDS] = {0};
  double prof_flops[NEGF_PROF_KINDS] = {0};
  int64_t prof_launches[NEGF_PROF_KINDS] = {0};

  // CUDA graph of the last call
  cudaGraphExec_t gexec = nullptr;
  bool have_key = false;
  CallKey key{};
};

namespace {

thread_local cudaError_t g_last_cuda = cudaSuccess;

inline negf_status cuda_status(cudaError_t e) {
  if (e != cudaSuccess) g_last_cuda = e;
  return e == cudaSuccess ? NEGF_OK : NEGF_ERR_CUDA;
}

#define NEGF_TRY(x)                                          \
  do {                                                       \
    cudaError_t _e = (x);                                    \
    if (_e != cudaSuccess) return _e;                        \
  } while (0)

#define NEGF_TRY_STATUS(x)                                   \
  do {                                                       \
    cudaError_t _e = (x);                                    \
    if (_e != cudaSuccess) return cuda_status(_e);           \
  } while (0)

int64_t sq(int x) { return (int64_t)x * x; }

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

  // Every kernel launch of the schedule goes through here so that the
  // optional profiler can bracket it with events on the launching stream.
  template <class F>
  cudaError_t launch(int kind, double flops, F f) {
    if (!p->profiling) return f();
    negf_plan_s::Rec r{kind, flops, nullptr, nullptr};
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
    if (g.bits == 0) g.bits = p->bits;
    if (p->precision == NEGF_MIXED)
      return launch(NEGF_PROF_GEMM_TC, gemm_flops(g), [&] { return negf::zgemm_tc(g, st); });
    return launch(NEGF_PROF_GEMM_F64, gemm_flops(g), [&] { return negf::zgemm_f64(g, st); });
  }
  cudaError_t gemm64(ZGemm g) {
    return launch(NEGF_PROF_GEMM_F64, gemm_flops(g), [&] { return negf::zgemm_f64(g, st); });
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

  // One step of iterative refinement of the last block column x = M^{-1} e_N
  // (mixed precision; gives G_1N = x_1 and T(E) to FP64-level accuracy):
  //   r = e_N - M x with FP64-accurate products (56-bit tensor-core split,
  //       exact integer accumulation, the E x term in FP64),
  //   d = L^{-1} D^{-1} U^{-1} r with the stored mixed factors, x <- x + d.
  // r / v live in the P region (free after last_column), q / d in RF.
  double2* RFblk(int i) const { return p->RF_ws + p->p_off[i] * p->chunk + (int64_t)wofs * p->b[i] * p->b[p->N - 1]; }
  cudaError_t refine_last_column() {
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
    for (int i = 0; i < N; ++i) {      // d = L^{-1} D^{-1} v, then x += d
      const int bi = p->b[i];
      ZGemm g;
      g.m = bi; g.n = bN; g.k = bi;
      g.A = Tblk(i); g.sA = sq(bi); g.lda = bi;
      g.B = Pblk(i); g.sB = (int64_t)bi * bN; g.ldb = bN;
      g.C = RFblk(i); g.sC = (int64_t)bi * bN; g.ldc = bN;
      g.batch = C;
      NEGF_TRY(gemm(g));
      for (int c = std::max(0, i - w); c < i; ++c) {
        ZGemm h;
        h.m = bi; h.n = bN; h.k = p->b[c];
        h.A = Xblk(i, c); h.sA = (int64_t)bi * p->b[c]; h.lda = p->b[c];
        h.B = RFblk(c); h.sB = (int64_t)p->b[c] * bN; h.ldb = bN;
        h.C = RFblk(i); h.sC = (int64_t)bi * bN; h.ldc = bN; h.alpha = {-1.0, 0.0};
        h.C1 = RFblk(i); h.sC1 = h.sC; h.ldc1 = bN; h.beta1 = {1.0, 0.0};
        h.batch = C;
        NEGF_TRY(gemm(h));
      }
    }
    for (int i = 0; i < N; ++i)
      NEGF_TRY(misc([&] {
        return negf::copy2d(RFblk(i), (int64_t)p->b[i] * bN, bN, LCblk(i), (int64_t)p->b[i] * bN, bN, p->b[i], bN,
                            1.0, 1, C, st);
      }));
    return cudaSuccess;
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

// ---------------------------------------------------------------------------
// Plan construction
// ---------------------------------------------------------------------------
negf_status validate(const negf_desc* d) {
  if (!d) return NEGF_ERR_ARG;
  if (d->n_blocks < 1 || !d->block_sizes) return NEGF_ERR_ARG;
  if (d->band_n < 3 || (d->band_n % 2) == 0) return NEGF_ERR_ARG;
  const int w = (d->band_n - 1) / 2;
  if (d->n_blocks <= w && d->n_blocks > 1) return NEGF_ERR_ARG;
  if (d->n_energies < 1) return NEGF_ERR_ARG;
  if (d->n_domains < 0 || (d->n_domains == 0 && d->domain_first_block)) return NEGF_ERR_ARG;
  if (d->precision != NEGF_FP64 && d->precision != NEGF_MIXED) return NEGF_ERR_ARG;
  if (d->refine_steps < 0 || d->refine_steps > 1) return NEGF_ERR_ARG;
  if (d->outputs & ~(NEGF_OUT_BAND | NEGF_OUT_G1N | NEGF_OUT_TRANSMISSION | NEGF_OUT_GRAD | NEGF_OUT_LESSER))
    return NEGF_ERR_ARG;
  if (d->checkpoint_every < 0) return NEGF_ERR_ARG;
  if (d->product_bits != 0 && (d->product_bits < 16 || d->product_bits > 56)) return NEGF_ERR_ARG;
  for (int i = 0; i < d->n_blocks; ++i)
    if (d->block_sizes[i] < 1 || d->block_sizes[i] > NEGF_MAX_BLOCK) return NEGF_ERR_ARG;
  return NEGF_OK;
}

}  // namespace

extern "C" {

const char* negf_status_string(negf_status s) {
  switch (s) {
    case NEGF_OK: return "NEGF_OK";
    case NEGF_ERR_ARG: return "NEGF_ERR_ARG: invalid argument";
    case NEGF_ERR_SINGULAR: return "NEGF_ERR_SINGULAR: zero pivot in a block inversion";
    case NEGF_ERR_NONFINITE: return "NEGF_ERR_NONFINITE: non-finite pivot in a block inversion";
    case NEGF_ERR_NOMEM: return "NEGF_ERR_NOMEM: workspace allocation failed";
    case NEGF_ERR_CUDA: return "NEGF_ERR_CUDA: CUDA runtime error";
    case NEGF_ERR_TIMEOUT: return "NEGF_ERR_TIMEOUT: bounded device wait expired";
    case NEGF_ERR_UNSUPPORTED: return "NEGF_ERR_UNSUPPORTED: not implemented for this descriptor";
  }
  return "negf: unknown status";
}

// RGF / DDRGF choice (n_domains = 0).  The batched sweep runs one CTA per
// block inversion; a layer step over x independent block problems costs
//     step(x; lat, thr) = max(lat, thr * x / slots)
// in units of one latency-bound plain-RGF layer step (slots: inversion CTAs
// resident on the GPU for the largest block).  Plain RGF: N steps over n_E
// problems, step(n_E; 1, 1).  DDRGF with d (D2, D1) pairs: N/d steps over the
// d n_E concurrent sub-domain problems with about 4.5x the launches of an
// RGF step (halo rows and columns, W / V, stitching) when latency-bound and
// about 15x its work when throughput-bound, then the interface RGF: d steps
// over n_E problems of w-layer super-blocks (w^3 the work).  The constants
// are fits to GB300 measurements (1024 x 64 and 4096 x 32 chains at 1, 8 and
// 64 energies, FP64 and mixed).  The cheapest d among 1 and the powers of
// two that leave pairs of at least 4w layers.
int32_t negf_auto_domains(int32_t n_blocks, const int32_t* block_sizes, int32_t band_n, int32_t n_energies,
                          int32_t sm_count) {
  if (n_blocks < 1 || !block_sizes || band_n < 3 || n_energies < 1 || sm_count < 1) return 1;
  const int w = (band_n - 1) / 2;
  int bmax = 1;
  for (int i = 0; i < n_blocks; ++i) bmax = std::max(bmax, (int)block_sizes[i]);
  // inversion CTAs per SM: shared memory (b (b+1) complex + 1 KB) and at most
  // five 256-thread CTAs (registers); blocks above 119 take a 2-SM cluster
  const double per_cta = (double)bmax * (bmax + 1) * 16.0 + 1024.0;
  const double slots = bmax <= 119 ? (double)sm_count * std::min(5.0, std::max(1.0, std::floor(233472.0 / per_cta)))
                                   : std::max(1.0, std::floor(sm_count / 2.0));
  auto step = [&](double x, double lat, double thr) { return std::max(lat, thr * x / slots); };
  double best = (double)n_blocks * step(n_energies, 1.0, 1.0);
  int best_d = 1;
  for (int d = 2; n_blocks / d >= 4 * w; d *= 2) {
    const double t = (double)n_blocks / d * step((double)n_energies * d, 4.5, 15.0) +
                     (double)d * step(n_energies, 1.0, 1.0) * w * w * w;
    if (t < best) { best = t; best_d = d; }
  }
  return best_d;
}

int32_t negf_plan_n_domains(const negf_plan_t* p) { return p ? p->n_domains : -1; }

negf_status negf_plan(negf_plan_t** out, const negf_desc* din, void* cuda_stream) {
  if (!out) return NEGF_ERR_ARG;
  *out = nullptr;
  negf_status v = validate(din);
  if (v != NEGF_OK) return v;
  negf_desc dd_auto = *din;
  const negf_desc* d = &dd_auto;
  if (dd_auto.n_domains == 0) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      sms = 152;
    }
    dd_auto.n_domains = (din->outputs & NEGF_OUT_GRAD)
                            ? 1
                            : negf_auto_domains(din->n_blocks, din->block_sizes, din->band_n, din->n_energies, sms);
  }
  const int w = (d->band_n - 1) / 2;
  if (d->n_domains > 1 && (d->outputs & NEGF_OUT_GRAD)) return NEGF_ERR_UNSUPPORTED;
  if (d->precision == NEGF_MIXED && !negf::zgemm_tc_available()) return NEGF_ERR_UNSUPPORTED;
  if ((d->outputs & NEGF_OUT_GRAD) && w != 1) return NEGF_ERR_UNSUPPORTED;
  if ((d->outputs & NEGF_OUT_LESSER) && (w != 1 || d->n_domains > 1 || (d->checkpoint_every > 0 && (d->outputs & NEGF_OUT_GRAD))))
    return NEGF_ERR_UNSUPPORTED;
  {
    cudaError_t ie = negf::kernels_init();
    if (ie != cudaSuccess) { g_last_cuda = ie; return NEGF_ERR_CUDA; }
  }
  for (int i = 0; i < d->n_blocks; ++i)
    if (d->block_sizes[i] > negf::zinv_max_block()) return NEGF_ERR_UNSUPPORTED;

  negf_plan_s* p = new (std::nothrow) negf_plan_s();
  if (!p) return NEGF_ERR_NOMEM;
  p->N = d->n_blocks; p->w = w; p->nE = d->n_energies; p->n_domains = d->n_domains;
  p->precision = d->precision; p->refine = d->refine_steps; p->outputs = d->outputs;
  p->ckpt = d->checkpoint_every;
  p->bits = d->product_bits;
  // DDRGF sub-domains are closed systems (broadened by eta only): near their
  // internal resonances the halo chains amplify product rounding by up to
  // ~1e7 (measured on the pentadiagonal 256 x 32 workload at eta = 1e-6), so
  // mixed DDRGF defaults to 56-bit products
  if (p->n_domains > 1 && p->precision == NEGF_MIXED && p->bits == 0) p->bits = 56;
  p->b.assign(d->block_sizes, d->block_sizes + d->n_blocks);
  p->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&p->device);
  const int N = p->N;

  // band-packed offsets: d = -w..w outer, i inner, existing blocks only
  p->band_off.assign((size_t)(2 * w + 1) * N, -1);
  int64_t off = 0;
  for (int dd = -w; dd <= w; ++dd)
    for (int i = 0; i < N; ++i) {
      int j = i + dd;
      if (j < 0 || j >= N) continue;
      p->band_off[(size_t)(dd + w) * N + i] = off;
      off += (int64_t)p->b[i] * p->b[j];
    }
  p->band_elems = off;

  // DDRGF domain layout (Fig. parallel_RGF_domains): pair j = D2_j then its
  // separator D1_j of w layers; D2 first, D1 last.  Default boundaries balance
  // the layer weights b_i^3 (Sec. 3, cost model paragraph on inhomogeneous
  // systems).
  int64_t dd_e = 0;
  if (p->n_domains > 1) {
    const int nd = p->n_domains;
    std::vector<int> first(nd);
    if (d->domain_first_block) {
      for (int j = 0; j < nd; ++j) first[j] = d->domain_first_block[j];
    } else {
      std::vector<double> cum(N + 1, 0.0);
      for (int i = 0; i < N; ++i) cum[i + 1] = cum[i] + (double)p->b[i] * p->b[i] * p->b[i];
      int i = 0;
      for (int j = 0; j < nd; ++j) {
        const double target = cum[N] * j / nd;
        while (i < N && cum[i] < target - 1e-9 * cum[N]) ++i;
        first[j] = j == 0 ? 0 : i;
      }
    }
    p->dom_f.resize(nd); p->dom_l.resize(nd);
    for (int j = 0; j < nd; ++j) {
      const int lo = first[j], hi = (j + 1 < nd) ? first[j + 1] : N;   // pair = [lo, hi)
      if ((j == 0 && lo != 0) || hi - lo < 2 * w || hi - lo - w < 1) { delete p; return NEGF_ERR_ARG; }
      p->dom_f[j] = lo;
      p->dom_l[j] = hi - w - 1;
    }
    p->dom_of.assign(N, -1); p->sep_of.assign(N, -1); p->off_in.assign(N, 0);
    p->Fsz.assign(nd, 0); p->Lsz.assign(nd, 0); p->Psz.assign(nd, 0);
    for (int j = 0; j < nd; ++j) {
      for (int a = p->dom_f[j]; a <= p->dom_l[j]; ++a) p->dom_of[a] = j;
      for (int r = 0; r < w; ++r) {
        p->Fsz[j] += p->b[p->dom_f[j] + r];
        p->Lsz[j] += p->b[p->dom_l[j] - w + 1 + r];
        const int sl = p->dom_l[j] + 1 + r;
        p->sep_of[sl] = j;
        p->off_in[sl] = p->Psz[j];
        p->Psz[j] += p->b[sl];
      }
      p->Pmax = std::max(p->Pmax, p->Psz[j]);
    }
    p->fc_off.assign(N, 0); p->lc_off.assign(N, 0); p->wp_off.assign(N, 0); p->wq_off.assign(N, 0);
    for (int a = 0; a < N; ++a) {
      const int j = p->dom_of[a];
      if (j < 0) continue;
      const int Pp = j > 0 ? p->Psz[j - 1] : 0;
      p->fc_off[a] = p->fc_e; p->fc_e += (int64_t)p->b[a] * p->Fsz[j];
      p->lc_off[a] = p->lc_e; p->lc_e += (int64_t)p->b[a] * p->Lsz[j];
      p->wp_off[a] = p->wp_e; p->wp_e += (int64_t)p->b[a] * Pp;
      p->wq_off[a] = p->wq_e; p->wq_e += (int64_t)p->b[a] * p->Psz[j];
    }
    p->tsd_off.assign(nd, 0); p->tsu_off.assign(nd, 0); p->rs_off.assign(nd, 0); p->ts_x_off.assign(nd, 0);
    for (int k = 0; k < nd; ++k) {
      p->tsd_off[k] = p->tsd_e; p->tsd_e += sq(p->Psz[k]);
      p->rs_off[k] = p->rs_e; p->rs_e += (int64_t)p->Psz[0] * p->Psz[k];
      if (k + 1 < nd) { p->tsu_off[k] = p->tsu_e; p->tsu_e += (int64_t)p->Psz[k] * p->Psz[k + 1]; }
      if (k >= 1) { p->ts_x_off[k] = p->ts_x_e; p->ts_x_e += (int64_t)p->Psz[k] * p->Psz[k - 1]; }
    }
    p->mfp_off.assign(nd, 0); p->mpf_off.assign(nd, 0); p->mlq_off.assign(nd, 0); p->mql_off.assign(nd, 0);
    for (int j = 0; j < nd; ++j) {
      const int Pp = j > 0 ? p->Psz[j - 1] : 0;
      p->mfp_off[j] = p->msup_e; p->msup_e += (int64_t)p->Fsz[j] * Pp;
      p->mpf_off[j] = p->msup_e; p->msup_e += (int64_t)Pp * p->Fsz[j];
      p->mlq_off[j] = p->msup_e; p->msup_e += (int64_t)p->Lsz[j] * p->Psz[j];
      p->mql_off[j] = p->msup_e; p->msup_e += (int64_t)p->Psz[j] * p->Lsz[j];
    }
    if (p->Pmax > negf::zinv_max_block()) { delete p; return NEGF_ERR_UNSUPPORTED; }
    dd_e = 2 * p->fc_e + 3 * p->lc_e + 3 * p->wp_e + 3 * p->wq_e + 3 * p->tsd_e + 4 * p->tsu_e +
           2 * p->ts_x_e + sq(p->Pmax) + p->rs_e + p->band_elems;
  }

  // per-energy workspace layout
  int bmax = *std::max_element(p->b.begin(), p->b.end());
  p->t_off.resize(N); p->x_off.assign((size_t)N * w, 0); p->y_off.assign((size_t)N * w, 0);
  int64_t te = 0, xe = 0, ye = 0;
  for (int i = 0; i < N; ++i) {
    p->t_off[i] = te; te += sq(p->b[i]);
    for (int c = std::max(0, i - w); c < i; ++c) {
      p->x_off[(size_t)i * w + (i - c - 1)] = xe; xe += (int64_t)p->b[i] * p->b[c];
      p->y_off[(size_t)i * w + (i - c - 1)] = ye; ye += (int64_t)p->b[c] * p->b[i];
    }
  }
  p->s_slot = sq(bmax);
  const bool grad = (d->outputs & NEGF_OUT_GRAD) != 0;
  const int bN = p->b[N - 1], b0 = p->b[0];
  p->bmax2 = sq(bmax);
  p->bmaxN = (int64_t)bmax * bN;
  if (grad && d->checkpoint_every > 0) {
    // rings of k + 1 layers with fixed per-energy strides, plus one
    // checkpoint (S_hi, P_hi) per segment of k layers
    p->ck_k = std::min(d->checkpoint_every, N);
    p->ck_nseg = (N + p->ck_k - 1) / p->ck_k;
    te = xe = ye = (int64_t)(p->ck_k + 1) * p->bmax2;
  }
  p->t_elems = te; p->x_elems = xe; p->y_elems = ye;
  p->full_row = grad && p->ck_k == 0;
  p->r_off.resize(N);
  int64_t re = 0;
  for (int j = 0; j < N; ++j) { p->r_off[j] = re; re += (int64_t)p->b[0] * p->b[j]; }
  p->r_elems = p->full_row ? re : bmax;   // ring: (w+1) slots of b0 x bmax
  p->p_off.resize(N);
  int64_t pe = 0;
  for (int i = 0; i < N; ++i) { p->p_off[i] = pe; pe += (int64_t)p->b[i] * bN; }
  const bool refine = d->refine_steps > 0 && d->precision == NEGF_MIXED && d->n_domains == 1 && p->ck_k == 0;
  p->refine = refine ? 1 : 0;
  p->p_elems = (grad || refine) ? pe : 0;
  int64_t rf_elems = refine ? pe : 0;
  int64_t ck_elems = 0;
  if (p->ck_k > 0) {
    p->p_elems = (int64_t)(p->ck_k + 1) * p->bmaxN;
    ck_elems = (int64_t)p->ck_nseg * (p->bmax2 + p->bmaxN);
  }
  // Gamma_L, Gamma_R, P, Q, G_1N, and two more b1 x bN temporaries (gradient)
  p->scr_elems = sq(b0) + sq(bN) + 5 * (int64_t)b0 * bN;

  const int64_t lesser_e = (d->outputs & NEGF_OUT_LESSER) ? 2 * te : 0;
  const int64_t dh_e = grad ? p->bmax2 : 0;
  int64_t per_e = dh_e + lesser_e + te + xe + ye + (int64_t)(w + 1) * (w + 1) * p->s_slot * std::max(1, p->n_domains) +
                  (p->full_row ? re : (int64_t)(w + 1) * b0 * bmax) + 2 * p->p_elems + rf_elems + ck_elems +
                  p->scr_elems + dd_e;
  // chunk energies so that the workspace stays within a budget: 45% of the
  // device memory free at plan time, at least 24 GiB (the caller's outputs
  // need the rest)
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); free_b = 0; }
  const double budget_bytes = std::max(24.0 * (1ull << 30), 0.45 * (double)free_b);
  const int64_t budget_elems = (int64_t)(budget_bytes / (double)sizeof(double2));
  int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(p->nE, budget_elems / std::max<int64_t>(per_e, 1)));
  p->chunk = chunk;
  p->ws_bytes = (size_t)(per_e * chunk + p->msup_e) * sizeof(double2) + 256;
  cudaError_t err = cudaMalloc((void**)&p->ws, p->ws_bytes);
  if (err != cudaSuccess) { g_last_cuda = err; cudaGetLastError(); delete p; return NEGF_ERR_NOMEM; }
  err = cudaMalloc((void**)&p->d_err, sizeof(int) + sizeof(double) * (size_t)p->nE);
  if (err != cudaSuccess) { cudaGetLastError(); cudaFree(p->ws); delete p; return NEGF_ERR_NOMEM; }
  cudaMemset(p->d_err, 0, sizeof(int));
  p->Tdummy = reinterpret_cast<double*>(p->d_err + 2);
  double2* q = reinterpret_cast<double2*>(p->ws);
  p->T_ws = q; q += te * chunk;
  p->X_ws = q; q += xe * chunk;
  p->Y_ws = q; q += ye * chunk;
  p->S_ws = q; q += (int64_t)(w + 1) * (w + 1) * p->s_slot * std::max(1, p->n_domains) * chunk;
  p->R_ws = q; q += (p->full_row ? re : (int64_t)(w + 1) * b0 * bmax) * chunk;
  p->P_ws = q; q += p->p_elems * chunk;
  p->LC_ws = q; q += p->p_elems * chunk;
  p->RF_ws = q; q += rf_elems * chunk;
  if (p->ck_k > 0) {
    p->CKS = q; q += (int64_t)p->ck_nseg * p->bmax2 * chunk;
    p->CKP = q; q += (int64_t)p->ck_nseg * p->bmaxN * chunk;
  }
  if (dh_e) {
    p->DH_ws = q; q += dh_e * chunk;
  }
  if (lesser_e) {
    p->LW_ws = q; q += te * chunk;
    p->LG_ws = q; q += te * chunk;
  }
  p->scratch = q; q += p->scr_elems * chunk;
  p->G1N_ws = p->scratch + (sq(b0) + sq(bN) + 2 * (int64_t)b0 * bN) * chunk;
  if (p->n_domains > 1) {
    p->FC = q; q += p->fc_e * chunk;
    p->FR = q; q += p->fc_e * chunk;
    p->LCd = q; q += p->lc_e * chunk;
    p->LR = q; q += p->lc_e * chunk;
    p->VT = q; q += p->lc_e * chunk;
    p->Wp = q; q += p->wp_e * chunk;
    p->Vp = q; q += p->wp_e * chunk;
    p->Zp = q; q += p->wp_e * chunk;
    p->Wq = q; q += p->wq_e * chunk;
    p->Vq = q; q += p->wq_e * chunk;
    p->Zq = q; q += p->wq_e * chunk;
    p->TSd = q; q += p->tsd_e * chunk;
    p->GSd = q; q += p->tsd_e * chunk;
    p->tS = q; q += p->tsd_e * chunk;
    p->TSu = q; q += p->tsu_e * chunk;
    p->TSl = q; q += p->tsu_e * chunk;
    p->GSu = q; q += p->tsu_e * chunk;
    p->GSl = q; q += p->tsu_e * chunk;
    p->XS = q; q += p->ts_x_e * chunk;
    p->YS = q; q += p->ts_x_e * chunk;
    p->SS = q; q += sq(p->Pmax) * chunk;
    p->RS = q; q += p->rs_e * chunk;
    p->band_ws = q; q += p->band_elems * chunk;
    p->Msup = q; q += p->msup_e;
  }
  // one-time kernel attributes (kept out of graph capture)
  {
    cudaError_t ie = negf::kernels_init();
    if (ie != cudaSuccess) { g_last_cuda = ie; negf_destroy(p); return NEGF_ERR_CUDA; }
  }
  {
    // energy groups: up to 4, with at least 128 energies each (fewer energies
    // leave each batched launch too small to fill the GPU)
    p->groups = std::max(1, std::min(4, p->chunk / 128));
    const char* env = getenv("NEGF_STREAMS");
    if (env) p->groups = std::max(1, std::min(NEGF_MAX_GROUPS, atoi(env)));
    p->groups = std::min(p->groups, p->chunk);
    // streams and events for up to NEGF_MAX_GROUPS groups (negf_autotune may
    // change the count); DDRGF plans keep the count fixed
    const int gcap = p->n_domains > 1 ? p->groups : std::max(p->groups, std::min(NEGF_MAX_GROUPS, p->chunk));
    for (int g = 1; g < gcap; ++g) {
      cudaStream_t s2 = nullptr;
      if (cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess) { negf_destroy(p); return NEGF_ERR_CUDA; }
      p->side.push_back(s2);
    }
    for (int g = 0; g < gcap; ++g) {
      cudaEvent_t e2 = nullptr, e3 = nullptr;
      if (cudaEventCreateWithFlags(&e2, cudaEventDisableTiming) != cudaSuccess) { negf_destroy(p); return NEGF_ERR_CUDA; }
      p->ev.push_back(e2);
      if (cudaEventCreateWithFlags(&e3, cudaEventDisableTiming) != cudaSuccess) { negf_destroy(p); return NEGF_ERR_CUDA; }
      p->stagger.push_back(e3);
    }
    if (p->n_domains > 1) {
      const int nd = p->n_domains;
      p->dstream.assign((size_t)p->groups * nd, nullptr);
      for (int g = 0; g < p->groups; ++g) {
        cudaEvent_t f = nullptr;
        if (cudaEventCreateWithFlags(&f, cudaEventDisableTiming) != cudaSuccess) { negf_destroy(p); return NEGF_ERR_CUDA; }
        p->dfork.push_back(f);
        for (int j = 0; j < nd; ++j) {
          cudaEvent_t jn = nullptr;
          if (cudaEventCreateWithFlags(&jn, cudaEventDisableTiming) != cudaSuccess) { negf_destroy(p); return NEGF_ERR_CUDA; }
          p->djoin.push_back(jn);
          if (j == 0) continue;
          if (cudaStreamCreateWithFlags(&p->dstream[(size_t)g * nd + j], cudaStreamNonBlocking) != cudaSuccess) {
            negf_destroy(p);
            return NEGF_ERR_CUDA;
          }
        }
      }
    }
  }
  *out = p;
  return NEGF_OK;
}

size_t negf_workspace_bytes(const negf_plan_t* p) { return p ? p->ws_bytes : 0; }

const char* negf_last_cuda_error(void) { return cudaGetErrorString(g_last_cuda); }

int64_t negf_band_offset(const negf_plan_t* p, int32_t d, int32_t i) {
  if (!p || d < -p->w || d > p->w || i < 0 || i >= p->N) return -1;
  return p->band_off[(size_t)(d + p->w) * p->N + i];
}

int64_t negf_band_elems(const negf_plan_t* p) { return p ? p->band_elems : -1; }

void negf_destroy(negf_plan_t* p) {
  if (!p) return;
  if (p->gexec) {
    cudaStreamSynchronize(p->stream);
    cudaGraphExecDestroy(p->gexec);
  }
  for (auto s2 : p->side) cudaStreamDestroy(s2);
  for (auto e2 : p->ev) cudaEventDestroy(e2);
  for (auto e3 : p->stagger) cudaEventDestroy(e3);
  for (auto s3 : p->dstream) if (s3) cudaStreamDestroy(s3);
  for (auto e4 : p->dfork) cudaEventDestroy(e4);
  for (auto e5 : p->djoin) cudaEventDestroy(e5);
  cudaFree(p->ws);
  cudaFree(p->d_err);
  if (p->host_io) cudaFree(p->host_io);
  delete p;
}

negf_status negf_sync(negf_plan_t* p) {
  if (!p) return NEGF_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return NEGF_ERR_CUDA;
  int word = 0;
  e = cudaMemcpy(&word, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return NEGF_ERR_CUDA;
  if (word) cudaMemset(p->d_err, 0, sizeof(int));
  if (word & negf::ERRBIT_NONFINITE) return NEGF_ERR_NONFINITE;
  if (word & negf::ERRBIT_SINGULAR) return NEGF_ERR_SINGULAR;
  if (word & negf::ERRBIT_TIMEOUT) return NEGF_ERR_TIMEOUT;
  return NEGF_OK;
}

}  // extern "C"

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

enum CallKind { CALL_SOLVE = 1, CALL_TRANS = 2, CALL_GRAD = 3 };

// Splits the energies [e0, e0 + ne) of one chunk into p->groups independent
// ranges, forks them onto the plan's side streams and joins them back, so
// that one range's block products run while another range inverts.
template <class F>
cudaError_t for_groups(negf_plan_s* p, Sweep base, F f, bool stagger = true) {
  const int G = std::min(p->groups, base.ne);
  if (G <= 1) return f(base);
  NEGF_TRY(cudaEventRecord(p->ev[0], p->stream));
  for (int g = 1; g < G; ++g) NEGF_TRY(cudaStreamWaitEvent(p->side[g - 1], p->ev[0], 0));
  for (int g = 0; g < G; ++g) {
    const int lo = (int)((int64_t)base.ne * g / G), hi = (int)((int64_t)base.ne * (g + 1) / G);
    Sweep s = base;
    s.st = g == 0 ? p->stream : p->side[g - 1];
    s.grp = g;
    s.e0 = base.e0 + lo;
    s.ne = hi - lo;
    s.wofs = base.wofs + lo;
    // Stagger: group g starts after the first inversion of group g-1, so
    // that one group's block products (tensor / integer pipes) run while the
    // next group inverts (FP64 pipe) instead of both alternating in step.
    if (stagger && g > 0) NEGF_TRY(cudaStreamWaitEvent(s.st, p->stagger[g - 1], 0));
    if (stagger && g + 1 < G) s.after_first_inv = p->stagger[g];
    NEGF_TRY(f(s));
  }
  for (int g = 1; g < G; ++g) {
    NEGF_TRY(cudaEventRecord(p->ev[g], p->side[g - 1]));
    NEGF_TRY(cudaStreamWaitEvent(p->stream, p->ev[g], 0));
  }
  return cudaSuccess;
}

// Drop the plan's executable graph.  Its last launch may still be running
// on the plan's stream, so the stream is drained first.
void drop_graph(negf_plan_s* p) {
  if (p->gexec) {
    cudaStreamSynchronize(p->stream);
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  p->have_key = false;
}

// Enqueue (or replay) the schedule of one call.  `body` enqueues the work of
// every energy chunk on p->stream.
template <class F>
negf_status run_captured(negf_plan_s* p, const CallKey& key, F body) {
  // Graph capture needs a created stream; on the legacy default stream, or
  // while profiling, the schedule is launched directly.
  if (p->profiling || p->stream == nullptr || p->stream == cudaStreamLegacy || p->stream == cudaStreamPerThread)
    return cuda_status(body());
  if (p->have_key && p->key == key && p->gexec) {
    return cuda_status(cudaGraphLaunch(p->gexec, p->stream));
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return NEGF_ERR_CUDA;
  cudaError_t be = body();
  e = cudaStreamEndCapture(p->stream, &graph);
  if (be != cudaSuccess || e != cudaSuccess) {
    g_last_cuda = be != cudaSuccess ? be : e;
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return NEGF_ERR_CUDA;
  }
  drop_graph(p);
  e = cudaGraphInstantiate(&p->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) { p->gexec = nullptr; p->have_key = false; return NEGF_ERR_CUDA; }
  p->key = key;
  p->have_key = true;
  return cuda_status(cudaGraphLaunch(p->gexec, p->stream));
}

}  // namespace

extern "C" {

negf_status negf_solve(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                       const negf_c128* sigma_R, int64_t sigma_E_stride, const negf_c128* E,
                       negf_c128* G_band, negf_c128* G_1N, int32_t* info) {
  if (!p || !H || !E || !info || sigma_E_stride < 0) return NEGF_ERR_ARG;
  if (!G_band && !G_1N) return NEGF_ERR_ARG;
  // a checkpointed adjoint plan keeps rings of k + 1 layers, not the whole
  // factorisation the band needs
  if (p->ck_k > 0 && G_band) return NEGF_ERR_UNSUPPORTED;
  CallKey key{};
  key.kind = CALL_SOLVE;
  key.stride = sigma_E_stride;
  const void* ptrs[] = {H, sigma_L, sigma_R, E, G_band, G_1N, info};
  std::memcpy(key.p, ptrs, sizeof(ptrs));
  return run_captured(p, key, [&]() -> cudaError_t {
    NEGF_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t) * p->nE, p->stream));
    for (int e0 = 0; e0 < p->nE; e0 += p->chunk) {
      Sweep base{p, p->stream, (const double2*)H, (const double2*)sigma_L, (const double2*)sigma_R,
                 sigma_E_stride, (const double2*)E, (double2*)G_band, (double2*)G_1N, info,
                 e0, std::min(p->chunk, p->nE - e0)};
      const int64_t s1 = (int64_t)p->b[0] * p->b[p->N - 1];
      if (p->n_domains > 1) {
        if (!G_band) { base.Gband = p->band_ws; base.gb_e0 = e0; }
        if (e0 == 0) NEGF_TRY(DD(p, base).assemble_msup());
        NEGF_TRY(for_groups(p, base, [&](Sweep& s) -> cudaError_t {
          return DD(p, s).run(true, G_1N ? (double2*)G_1N + (int64_t)s.e0 * s1 : nullptr, s1);
        }));
        continue;
      }
      NEGF_TRY(for_groups(p, base, [&](Sweep& s) -> cudaError_t {
        if (p->ck_k > 0) return s.ck_forward((double2*)G_1N + (int64_t)s.e0 * s1, s1);
        NEGF_TRY(s.upward(G_band != nullptr || (G_1N && p->refine)));
        if (G_band) NEGF_TRY(s.downward());
        if (G_1N && p->refine) {   // G_1N = first block of the refined last column
          NEGF_TRY(s.last_column());
          NEGF_TRY(s.refine_last_column());
          return s.misc([&] {
            return negf::copy_blocks(s.LCblk(0), s1, (double2*)G_1N + (int64_t)s.e0 * s1, s1, s1, s.ne, s.st);
          });
        }
        if (G_1N) NEGF_TRY(s.first_row((double2*)G_1N + (int64_t)s.e0 * s1, s1));
        return cudaSuccess;
      }));
    }
    return cudaSuccess;
  });
}

negf_status negf_transmission(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                              const negf_c128* sigma_R, int64_t sigma_E_stride, const negf_c128* E,
                              double* T, int32_t* info) {
  if (!p || !H || !E || !info || !T || !sigma_L || !sigma_R || sigma_E_stride < 0) return NEGF_ERR_ARG;
  CallKey key{};
  key.kind = CALL_TRANS;
  key.stride = sigma_E_stride;
  const void* ptrs[] = {H, sigma_L, sigma_R, E, T, info};
  std::memcpy(key.p, ptrs, sizeof(ptrs));
  return run_captured(p, key, [&]() -> cudaError_t {
    NEGF_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t) * p->nE, p->stream));
    const int64_t s1 = (int64_t)p->b[0] * p->b[p->N - 1];
    for (int e0 = 0; e0 < p->nE; e0 += p->chunk) {
      Sweep base{p, p->stream, (const double2*)H, (const double2*)sigma_L, (const double2*)sigma_R,
                 sigma_E_stride, (const double2*)E, nullptr, nullptr, info,
                 e0, std::min(p->chunk, p->nE - e0)};
      if (p->n_domains > 1) {
        base.Gband = p->band_ws;
        base.gb_e0 = e0;
        if (e0 == 0) NEGF_TRY(DD(p, base).assemble_msup());
      }
      NEGF_TRY(for_groups(p, base, [&](Sweep& s) -> cudaError_t {
        double2* g1n = p->G1N_ws + (int64_t)s.wofs * s1;
        if (p->n_domains > 1) {
          NEGF_TRY(DD(p, s).run(false, g1n, s1));
        } else if (p->ck_k > 0) {      // checkpointed plan: G_1N = t_1 (U^{-1} e_N)_1
          NEGF_TRY(s.ck_forward(g1n, s1));
        } else if (p->refine) {
          NEGF_TRY(s.upward(true));
          NEGF_TRY(s.last_column());
          NEGF_TRY(s.refine_last_column());
          NEGF_TRY(s.misc([&] { return negf::copy_blocks(s.LCblk(0), s1, g1n, s1, s1, s.ne, s.st); }));
        } else {
          NEGF_TRY(s.upward(false));
          NEGF_TRY(s.first_row(g1n, s1));
        }
        return s.transmission(g1n, s1, T);
      }));
    }
    return cudaSuccess;
  });
}

negf_status negf_grad(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                      const negf_c128* sigma_R, int64_t sigma_E_stride, const negf_c128* E,
                      const double* dL_dT, double* T, negf_c128* dH, negf_c128* dSigma_L,
                      negf_c128* dSigma_R, int32_t* info) {
  if (!p || !H || !E || !info || !dL_dT || !dH || !sigma_L || !sigma_R || sigma_E_stride < 0) return NEGF_ERR_ARG;
  if (!(p->outputs & NEGF_OUT_GRAD)) return NEGF_ERR_ARG;
  CallKey key{};
  key.kind = CALL_GRAD;
  key.stride = sigma_E_stride;
  const void* ptrs[] = {H, sigma_L, sigma_R, E, dL_dT, T, dH, dSigma_L, dSigma_R, info};
  std::memcpy(key.p, ptrs, sizeof(ptrs));
  const int N = p->N, b0 = p->b[0], bN = p->b[N - 1];
  const int64_t s1 = (int64_t)b0 * bN;
  const bool ck = p->ck_k > 0;
  return run_captured(p, key, [&]() -> cudaError_t {
    NEGF_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t) * p->nE, p->stream));
    for (int e0 = 0; e0 < p->nE; e0 += p->chunk) {
      const int ne = std::min(p->chunk, p->nE - e0);
      const bool first = (e0 == 0);
      Sweep base{p, p->stream, (const double2*)H, (const double2*)sigma_L, (const double2*)sigma_R,
                 sigma_E_stride, (const double2*)E, nullptr, nullptr, info, e0, ne};
      Sweep s = base;   // wofs = 0: the whole chunk, for the energy-reduced products

      // dH_ab (+)= 2 sum_e w_e (G_{b,N} U_a)^H: the per-energy products
      // P_e = G_{b,N} U_a batched over the chunk (plan precision), then their
      // weighted, conjugate-transposed sum over energies
      auto dh_pair = [&](int a, int bb, const double2* Ua, int64_t sUa, const double2* Lb, int64_t sLb) {
        const int ba = p->b[a], bbs = p->b[bb];
        double2* out = (double2*)dH + p->band_off[(size_t)(bb - a + p->w) * N + a];
        ZGemm g;
        g.m = bbs; g.n = ba; g.k = bN;
        g.A = Lb; g.sA = sLb; g.lda = bN;
        g.B = Ua; g.sB = sUa; g.ldb = ba;
        g.C = p->DH_ws; g.sC = p->bmax2; g.ldc = ba;
        g.batch = ne;
        NEGF_TRY(s.gemm(g));
        return s.misc([&] {
          return negf::reduce_energies(p->DH_ws, p->bmax2, ba, ne, dL_dT + e0, out, bbs, ba, bbs, {2.0, 0.0},
                                       first ? 0 : 1, 1, p->stream);
        });
      };
      // per-energy Sigma: the M-path part 2 w_e (G_{i,N} U_i)^H of layer 0 / N-1
      auto sigma_mpath = [&](int side, const double2* Ui, int64_t sUi, const double2* Li, int64_t sLi) {
        negf_c128* dS = side == 0 ? dSigma_L : dSigma_R;
        if (!dS || sigma_E_stride == 0) return cudaSuccess;
        const int bs = side == 0 ? b0 : bN;
        ZGemm h;
        h.m = bs; h.n = bs; h.k = bN;
        h.A = Ui; h.sA = sUi; h.lda = bs; h.opA = negf::OP_C;
        h.B = Li; h.sB = sLi; h.ldb = bN; h.opB = negf::OP_C;
        h.C = (double2*)dS + (int64_t)e0 * sigma_E_stride; h.sC = sigma_E_stride; h.ldc = bs;
        h.alpha = {2.0, 0.0}; h.weight = dL_dT + e0; h.batch = ne;
        return s.gemm64(h);
      };

      if (!ck) {
        NEGF_TRY(for_groups(p, base, [&](Sweep& sw) -> cudaError_t {
          double2* g1n = sw.scr(4);
          NEGF_TRY(sw.upward(true));
          NEGF_TRY(sw.first_row(g1n, s1));
          NEGF_TRY(sw.last_column());
          if (T) NEGF_TRY(sw.transmission(g1n, s1, T));
          return sw.grad_prep(g1n, s1);
        }));
        for (int a = 0; a < N; ++a)
          for (int bb = std::max(0, a - 1); bb <= std::min(N - 1, a + 1); ++bb)
            NEGF_TRY(dh_pair(a, bb, s.Pblk(a), (int64_t)p->b[a] * bN, s.LCblk(bb), (int64_t)p->b[bb] * bN));
        NEGF_TRY(sigma_mpath(0, s.Pblk(0), s1, s.LCblk(0), s1));
        NEGF_TRY(sigma_mpath(1, s.Pblk(N - 1), sq(bN), s.LCblk(N - 1), sq(bN)));
      } else {
        // checkpointed: forward sweep with checkpoints, then segment by
        // segment (increasing layers) recompute, chains and reductions
        NEGF_TRY(for_groups(p, base, [&](Sweep& sw) -> cudaError_t {
          double2* g1n = sw.scr(4);
          NEGF_TRY(sw.ck_forward(g1n, s1));
          if (T) NEGF_TRY(sw.transmission(g1n, s1, T));
          return sw.grad_K(g1n, s1);
        }));
        for (int sg = 0; sg < p->ck_nseg; ++sg) {
          NEGF_TRY(for_groups(p, base, [&](Sweep& sw) -> cudaError_t {
            if (sg > 0) NEGF_TRY(sw.ck_recompute(sg));
            return sw.ck_chains(sg);
          }, sg > 0));
          const int lo = s.seg_lo(sg), hi = s.seg_hi(sg);
          for (int i = lo; i <= hi; ++i) {
            NEGF_TRY(dh_pair(i, i, s.cP(i), p->bmaxN, s.cL(i), p->bmaxN));
            if (i > 0) {
              NEGF_TRY(dh_pair(i - 1, i, s.cP(i - 1), p->bmaxN, s.cL(i), p->bmaxN));
              NEGF_TRY(dh_pair(i, i - 1, s.cP(i), p->bmaxN, s.cL(i - 1), p->bmaxN));
            }
          }
          if (lo == 0) NEGF_TRY(sigma_mpath(0, s.cP(0), p->bmaxN, s.cL(0), p->bmaxN));
          if (hi == N - 1) NEGF_TRY(sigma_mpath(1, s.cP(N - 1), p->bmaxN, s.cL(N - 1), p->bmaxN));
        }
      }
      // Sigma terms.  Sigma enters M like H (the X_11 / X_NN parts are the
      // dH_00 / dH_NN products) and also Gamma = i (Sigma - Sigma^H):
      //   dSigma_L (+)= -2i sum_e w_e G_1N Gamma_R G_1N^H,
      //   dSigma_R (+)= -2i sum_e w_e G_1N^H Gamma_L G_1N.
      for (int side = 0; side < 2; ++side) {
        negf_c128* dS = side == 0 ? dSigma_L : dSigma_R;
        if (!dS) continue;
        const int bs = side == 0 ? b0 : bN;
        double2* V = s.scr(5);   // V = Gamma_R G_1N^H (bN x b0) or Gamma_L G_1N (b0 x bN)
        {
          ZGemm g;
          if (side == 0) {
            g.m = bN; g.n = b0; g.k = bN;
            g.A = s.scr(1); g.sA = sigma_E_stride ? sq(bN) : 0; g.lda = bN;
            g.B = s.scr(4); g.sB = s1; g.ldb = bN; g.opB = negf::OP_C;
            g.C = V; g.sC = s1; g.ldc = b0;
          } else {
            g.m = b0; g.n = bN; g.k = b0;
            g.A = s.scr(0); g.sA = sigma_E_stride ? sq(b0) : 0; g.lda = b0;
            g.B = s.scr(4); g.sB = s1; g.ldb = bN;
            g.C = V; g.sC = s1; g.ldc = bN;
          }
          g.batch = ne;
          NEGF_TRY(s.gemm64(g));
        }
        ZGemm g;   // -2i sum_e w_e A_e or per energy
        if (side == 0) {
          g.m = b0; g.n = b0; g.k = bN;
          g.A = s.scr(4); g.sA = s1; g.lda = bN;
          g.B = V; g.sB = s1; g.ldb = b0;
        } else {
          g.m = bN; g.n = bN; g.k = b0;
          g.A = s.scr(4); g.sA = s1; g.lda = bN; g.opA = negf::OP_C;
          g.B = V; g.sB = s1; g.ldb = bN;
        }
        g.batch = ne;
        if (sigma_E_stride == 0) {   // per-energy products, then their weighted sum times -2i
          g.C = p->DH_ws; g.sC = p->bmax2; g.ldc = bs;
          NEGF_TRY(s.gemm64(g));
          NEGF_TRY(s.misc([&] {
            return negf::reduce_energies(p->DH_ws, p->bmax2, bs, ne, dL_dT + e0, (double2*)dS, bs, bs, bs,
                                         {0.0, -2.0}, first ? 0 : 1, 0, p->stream);
          }));
        } else {   // per energy, onto the M-path part written above
          double2* out = (double2*)dS + (int64_t)e0 * sigma_E_stride;
          g.alpha = {0.0, -2.0};
          g.weight = dL_dT + e0;
          g.C = out; g.sC = sigma_E_stride; g.ldc = bs;
          g.C1 = out; g.sC1 = sigma_E_stride; g.ldc1 = bs; g.beta1 = {1.0, 0.0};
          NEGF_TRY(s.gemm64(g));
        }
      }
    }
    if (sigma_E_stride == 0) {   // add the M-path parts dH_00 / dH_NN once, after all chunks
      Sweep s{p, p->stream, nullptr, nullptr, nullptr, 0, nullptr, nullptr, nullptr, info, 0, 1};
      for (int side = 0; side < 2; ++side) {
        negf_c128* dS = side == 0 ? dSigma_L : dSigma_R;
        if (!dS) continue;
        const int layer = side == 0 ? 0 : N - 1, bs = p->b[layer];
        ZGemm g;
        g.m = bs; g.n = bs; g.k = 0;
        g.A = (double2*)dS; g.B = (double2*)dS; g.lda = bs; g.ldb = bs;
        g.C = (double2*)dS; g.ldc = bs;
        g.C1 = (double2*)dS; g.ldc1 = bs; g.beta1 = {1.0, 0.0};
        g.C2 = (const double2*)dH + p->band_off[(size_t)p->w * N + layer]; g.ldc2 = bs; g.beta2 = {1.0, 0.0};
        g.batch = 1;
        NEGF_TRY(s.gemm64(g));
      }
    }
    return cudaSuccess;
  });
}

}  // extern "C"

extern "C" {

// negf_solve from host memory to host memory: inputs copied to device
// buffers the plan owns, the captured solve, outputs copied back, all on the
// plan's stream; returns after the outputs are in host memory (with
// negf_sync's status).
negf_status negf_solve_host(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                            const negf_c128* sigma_R, int64_t sigma_E_stride, const negf_c128* E,
                            negf_c128* G_band, negf_c128* G_1N, int32_t* info) {
  if (!p || !H || !E || !info || sigma_E_stride < 0 || (!G_band && !G_1N)) return NEGF_ERR_ARG;
  const int64_t nE = p->nE, b0 = p->b[0], bN = p->b[p->N - 1];
  const int64_t nsig_L = sigma_E_stride ? (nE - 1) * sigma_E_stride + b0 * b0 : b0 * b0;
  const int64_t nsig_R = sigma_E_stride ? (nE - 1) * sigma_E_stride + bN * bN : bN * bN;
  auto al = [](int64_t elems) { return (size_t)((elems * (int64_t)sizeof(double2) + 255) / 256 * 256); };
  const size_t oH = 0, oL = oH + al(p->band_elems), oR = oL + al(nsig_L), oE = oR + al(nsig_R),
               oG = oE + al(nE), o1 = oG + al(nE * p->band_elems), oI = o1 + al(nE * b0 * bN),
               need = oI + al(nE);
  if (!p->host_io || p->host_io_bytes < need) {
    if (p->host_io) cudaFree(p->host_io);
    p->host_io = nullptr;
    p->host_io_bytes = 0;
    cudaError_t e = cudaMalloc((void**)&p->host_io, need);
    if (e != cudaSuccess) { g_last_cuda = e; cudaGetLastError(); return NEGF_ERR_NOMEM; }
    p->host_io_bytes = need;
  }
  char* d = p->host_io;
  negf_c128* dH = (negf_c128*)(d + oH);
  negf_c128* dL = sigma_L ? (negf_c128*)(d + oL) : nullptr;
  negf_c128* dR = sigma_R ? (negf_c128*)(d + oR) : nullptr;
  negf_c128* dE = (negf_c128*)(d + oE);
  negf_c128* dG = G_band ? (negf_c128*)(d + oG) : nullptr;
  negf_c128* d1 = G_1N ? (negf_c128*)(d + o1) : nullptr;
  int32_t* dI = (int32_t*)(d + oI);
  const size_t z = sizeof(negf_c128);
  cudaStream_t st = p->stream;
  cudaError_t e = cudaMemcpyAsync(dH, H, (size_t)p->band_elems * z, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && dL) e = cudaMemcpyAsync(dL, sigma_L, (size_t)nsig_L * z, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && dR) e = cudaMemcpyAsync(dR, sigma_R, (size_t)nsig_R * z, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dE, E, (size_t)nE * z, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e);
  negf_status s = negf_solve(p, dH, dL, dR, sigma_E_stride, dE, dG, d1, dI);
  if (s != NEGF_OK) return s;
  if (G_band) e = cudaMemcpyAsync(G_band, dG, (size_t)(nE * p->band_elems) * z, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && G_1N) e = cudaMemcpyAsync(G_1N, d1, (size_t)(nE * b0 * bN) * z, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(info, dI, (size_t)nE * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_status(e);
  return negf_sync(p);
}

// Keldysh equation for the selected blocks (see Sweep::lesser_up / down).
negf_status negf_lesser(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L, const negf_c128* sigma_R,
                        int64_t sigma_E_stride, const negf_c128* E, const negf_c128* sigma_less_L,
                        const negf_c128* sigma_less_R, int64_t sless_stride, const negf_c128* less_diag,
                        negf_c128* G_band, negf_c128* G_less, int32_t* info) {
  if (!p || !H || !E || !info || !G_band || !G_less || sigma_E_stride < 0 || sless_stride < 0) return NEGF_ERR_ARG;
  if (!(p->outputs & NEGF_OUT_LESSER)) return NEGF_ERR_ARG;
  CallKey key{};
  key.kind = 4;
  key.stride = sigma_E_stride * 1000003 + sless_stride;
  const void* ptrs[] = {H, sigma_L, sigma_R, E, sigma_less_L, sigma_less_R, less_diag, G_band, G_less, info};
  std::memcpy(key.p, ptrs, sizeof(ptrs));
  return run_captured(p, key, [&]() -> cudaError_t {
    NEGF_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t) * p->nE, p->stream));
    for (int e0 = 0; e0 < p->nE; e0 += p->chunk) {
      Sweep base{p, p->stream, (const double2*)H, (const double2*)sigma_L, (const double2*)sigma_R,
                 sigma_E_stride, (const double2*)E, (double2*)G_band, nullptr, info,
                 e0, std::min(p->chunk, p->nE - e0)};
      NEGF_TRY(for_groups(p, base, [&](Sweep& s) -> cudaError_t {
        NEGF_TRY(s.upward(true));
        NEGF_TRY(s.downward());
        NEGF_TRY(s.lesser_up((const double2*)sigma_less_L, (const double2*)sigma_less_R, sless_stride,
                             (const double2*)less_diag));
        return s.lesser_down((double2*)G_less);
      }));
    }
    return cudaSuccess;
  });
}

// Diagonal blocks of M G - I from the band alone (the check of a band that
// needs no off-band block): R_i = sum_{|c - i| <= w} M_{i,c} G_{c,i} - I,
// res[e] = sqrt(sum_i ||R_i||_F^2 / sum_i b_i), FP64 products.
negf_status negf_band_residual(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                               const negf_c128* sigma_R, int64_t sigma_E_stride, const negf_c128* E,
                               const negf_c128* G_band, double* res) {
  if (!p || !H || !E || !G_band || !res || sigma_E_stride < 0) return NEGF_ERR_ARG;
  const int N = p->N, w = p->w;
  int64_t sumb = 0;
  for (int i = 0; i < N; ++i) sumb += p->b[i];
  for (int e0 = 0; e0 < p->nE; e0 += p->chunk) {
    const int ne = std::min(p->chunk, p->nE - e0);
    Sweep s{p, p->stream, (const double2*)H, (const double2*)sigma_L, (const double2*)sigma_R, sigma_E_stride,
            (const double2*)E, (double2*)G_band, nullptr, nullptr, e0, ne};
    double2* R = s.Sslot(0, 0);
    const int64_t sRr = s.sS(), sG = p->band_elems;
    for (int i = 0; i < N; ++i) {
      const int bi = p->b[i];
      bool first = true;
      for (int c = std::max(0, i - w); c <= std::min(N - 1, i + w); ++c) {   // R (+)= -H_{i,c} G_{c,i}
        ZGemm g;
        g.m = bi; g.n = bi; g.k = p->b[c];
        g.A = s.Hblk(i, c); g.sA = 0; g.lda = p->b[c];
        g.B = s.Gb(c, i); g.sB = sG; g.ldb = bi;
        g.C = R; g.sC = sRr; g.ldc = bi; g.alpha = {-1.0, 0.0};
        if (!first) { g.C1 = R; g.sC1 = sRr; g.ldc1 = bi; g.beta1 = {1.0, 0.0}; }
        g.batch = ne;
        NEGF_TRY_STATUS(s.gemm64(g));
        first = false;
      }
      NEGF_TRY_STATUS(negf::axpy_scalar(R, sRr, s.Gb(i, i), sG, s.E + e0, 1.0, bi, bi, bi, ne, p->stream));
      for (int side = 0; side < 2; ++side) {   // - Sigma G_ii on the lead layers
        const double2* sg = side == 0 ? (i == 0 ? s.sigmaL() : nullptr) : (i == N - 1 ? s.sigmaR() : nullptr);
        if (!sg) continue;
        ZGemm g;
        g.m = bi; g.n = bi; g.k = bi;
        g.A = sg; g.sA = sigma_E_stride; g.lda = bi;
        g.B = s.Gb(i, i); g.sB = sG; g.ldb = bi;
        g.C = R; g.sC = sRr; g.ldc = bi; g.alpha = {-1.0, 0.0};
        g.C1 = R; g.sC1 = sRr; g.ldc1 = bi; g.beta1 = {1.0, 0.0};
        g.batch = ne;
        NEGF_TRY_STATUS(s.gemm64(g));
      }
      NEGF_TRY_STATUS(negf::add_diag(R, sRr, bi, bi, nullptr, 0, -1.0, ne, p->stream));
      NEGF_TRY_STATUS(negf::frob2(R, sRr, sq(bi), res + e0, ne, i > 0, p->stream));
    }
    NEGF_TRY_STATUS(negf::sqrt_scale(res + e0, ne, 1.0 / (double)sumb, p->stream));
  }
  return NEGF_OK;
}

// Energy-group autotuner: replays the plan's solve schedule with 1, 2, 3, 4,
// 6, 8 groups (those the plan's streams allow), times each with CUDA events
// on the plan's stream, and keeps the fastest.
negf_status negf_autotune(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L, const negf_c128* sigma_R,
                          int64_t sigma_E_stride, const negf_c128* E, negf_c128* G_band, negf_c128* G_1N,
                          int32_t* info, int32_t reps, int32_t* best_groups, double* ms) {
  if (!p || reps < 1) return NEGF_ERR_ARG;
  if (p->n_domains > 1 || p->ck_k > 0) return NEGF_ERR_UNSUPPORTED;
  const int cand[NEGF_AUTOTUNE_CANDIDATES] = {1, 2, 3, 4, 6, 8};
  const int gmax = (int)p->side.size() + 1;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return NEGF_ERR_CUDA;
  const int g0 = p->groups;
  int best = g0;
  double best_ms = 1e300;
  negf_status st = NEGF_OK;
  for (int k = 0; k < NEGF_AUTOTUNE_CANDIDATES; ++k) {
    if (ms) ms[k] = -1.0;
    const int G = cand[k];
    if (G > gmax) continue;
    p->groups = G;
    drop_graph(p);
    st = negf_solve(p, H, sigma_L, sigma_R, sigma_E_stride, E, G_band, G_1N, info);   // capture + warm-up
    if (st != NEGF_OK) break;
    if (cudaEventRecord(a, p->stream) != cudaSuccess) { st = NEGF_ERR_CUDA; break; }
    for (int r = 0; r < reps && st == NEGF_OK; ++r)
      st = negf_solve(p, H, sigma_L, sigma_R, sigma_E_stride, E, G_band, G_1N, info);
    if (st != NEGF_OK) break;
    float t = 0.0f;
    if (cudaEventRecord(b, p->stream) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
        cudaEventElapsedTime(&t, a, b) != cudaSuccess) { st = NEGF_ERR_CUDA; break; }
    const double per = (double)t / reps;
    if (ms) ms[k] = per;
    if (per < best_ms) { best_ms = per; best = G; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  p->groups = st == NEGF_OK ? best : g0;
  drop_graph(p);
  if (best_groups) *best_groups = p->groups;
  return st;
}

int32_t negf_plan_groups(const negf_plan_t* p) { return p ? p->groups : -1; }

negf_status negf_plan_set_groups(negf_plan_t* p, int32_t groups) {
  if (!p || groups < 1 || groups > (int)p->side.size() + 1) return NEGF_ERR_ARG;
  if (groups != p->groups) {
    if (p->n_domains > 1) return NEGF_ERR_UNSUPPORTED;   // per-group domain streams are fixed
    p->groups = groups;
    drop_graph(p);
  }
  return NEGF_OK;
}

negf_status negf_profile_enable(negf_plan_t* p, int32_t on) {
  if (!p) return NEGF_ERR_ARG;
  p->profiling = on != 0;
  return NEGF_OK;
}

int32_t negf_profile_read(negf_plan_t* p, double* ms, double* flops, int64_t* launches) {
  if (!p) return -1;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return -1;
  for (auto& r : p->recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      p->prof_ms[r.kind] += t;
      p->prof_flops[r.kind] += r.flops;
      p->prof_launches[r.kind] += 1;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  p->recs.clear();
  for (int k = 0; k < NEGF_PROF_KINDS; ++k) {
    if (ms) ms[k] = p->prof_ms[k];
    if (flops) flops[k] = p->prof_flops[k];
    if (launches) launches[k] = p->prof_launches[k];
    p->prof_ms[k] = 0; p->prof_flops[k] = 0; p->prof_launches[k] = 0;
  }
  return NEGF_PROF_KINDS;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// negf_solve_noalloc: negf_solve for callers that cannot allocate device
// memory.  The sweep's scratch lives in one file-scope device array that
// every GPU loading this library holds until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

static __device__ __align__(256) unsigned char g_noalloc_scratch[NEGF_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
// Device address of g_noalloc_scratch per device ordinal.  The host-side
// symbol g_noalloc_scratch is only a stand-in: kernels must receive this.
void* g_noalloc_base[kNoallocMaxDevices] = {};
}  // namespace

extern "C" negf_status negf_solve_noalloc(const negf_desc* d, const negf_c128* H, const negf_c128* sigma_L,
                                          const negf_c128* sigma_R, int64_t sigma_E_stride, const negf_c128* E,
                                          negf_c128* G_band, negf_c128* G_1N, int32_t* info, void* cuda_stream) {
  negf_status v = validate(d);
  if (v != NEGF_OK) return v;
  if (!H || !E || !info || sigma_E_stride < 0 || (!G_band && !G_1N)) return NEGF_ERR_ARG;
  if (d->n_domains != 1 || d->precision != NEGF_FP64 || (d->outputs & NEGF_OUT_GRAD)) return NEGF_ERR_UNSUPPORTED;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { g_last_cuda = e; return NEGF_ERR_CUDA; }
  if (dev < 0 || dev >= kNoallocMaxDevices) return NEGF_ERR_UNSUPPORTED;
  void* base = nullptr;
  {
    // One-time set-up per device, with that device current (first call).
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) { g_last_cuda = e; return NEGF_ERR_CUDA; }
      e = negf::kernels_init();
      if (e != cudaSuccess) { g_last_cuda = e; return NEGF_ERR_CUDA; }
      g_noalloc_base[dev] = ptr;
    }
    base = g_noalloc_base[dev];
  }
  const int w = (d->band_n - 1) / 2;
  for (int i = 0; i < d->n_blocks; ++i)
    if (d->block_sizes[i] > negf::zinv_max_block()) return NEGF_ERR_UNSUPPORTED;

  // Host-side layout of the same schedule as a plan, all energies in one
  // chunk, with every workspace region placed inside the static scratch.
  negf_plan_s p;
  p.N = d->n_blocks; p.w = w; p.nE = d->n_energies; p.n_domains = 1;
  p.precision = NEGF_FP64; p.refine = 0; p.outputs = d->outputs; p.ckpt = 0;
  p.b.assign(d->block_sizes, d->block_sizes + d->n_blocks);
  p.stream = (cudaStream_t)cuda_stream;
  p.device = dev;
  const int N = p.N;
  p.band_off.assign((size_t)(2 * w + 1) * N, -1);
  int64_t off = 0;
  for (int dd = -w; dd <= w; ++dd)
    for (int i = 0; i < N; ++i) {
      int j = i + dd;
      if (j < 0 || j >= N) continue;
      p.band_off[(size_t)(dd + w) * N + i] = off;
      off += (int64_t)p.b[i] * p.b[j];
    }
  p.band_elems = off;
  const int bmax = *std::max_element(p.b.begin(), p.b.end());
  p.t_off.resize(N); p.x_off.assign((size_t)N * w, 0); p.y_off.assign((size_t)N * w, 0);
  int64_t te = 0, xe = 0, ye = 0;
  for (int i = 0; i < N; ++i) {
    p.t_off[i] = te; te += sq(p.b[i]);
    for (int c = std::max(0, i - w); c < i; ++c) {
      p.x_off[(size_t)i * w + (i - c - 1)] = xe; xe += (int64_t)p.b[i] * p.b[c];
      p.y_off[(size_t)i * w + (i - c - 1)] = ye; ye += (int64_t)p.b[c] * p.b[i];
    }
  }
  p.s_slot = sq(bmax);
  p.r_elems = bmax;
  const int64_t ring = (int64_t)(w + 1) * p.b[0] * bmax;
  const int64_t per_e = te + xe + ye + (int64_t)(w + 1) * (w + 1) * p.s_slot + ring;
  const int64_t C = p.nE;
  const size_t need = 256 + (size_t)per_e * (size_t)C * sizeof(double2);
  if (need > (size_t)NEGF_NOALLOC_SCRATCH_BYTES) return NEGF_ERR_ARG;
  p.chunk = (int)C;
  p.d_err = reinterpret_cast<int*>(base);                      // first 256 bytes: error word
  double2* q = reinterpret_cast<double2*>(static_cast<char*>(base) + 256);
  p.T_ws = q; q += te * C;
  p.X_ws = q; q += xe * C;
  p.Y_ws = q; q += ye * C;
  p.S_ws = q; q += (int64_t)(w + 1) * (w + 1) * p.s_slot * C;
  p.R_ws = q;

  // The scratch keeps the previous call's contents: only the error word must
  // start at zero (every workspace block is written before it is read).
  cudaStream_t st = p.stream;
  e = cudaMemsetAsync(p.d_err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(info, 0, sizeof(int32_t) * (size_t)p.nE, st);
  if (e == cudaSuccess) {
    Sweep s{&p, st, (const double2*)H, (const double2*)sigma_L, (const double2*)sigma_R, sigma_E_stride,
            (const double2*)E, (double2*)G_band, (double2*)G_1N, info, 0, p.nE};
    e = s.upward(G_band != nullptr);
    if (e == cudaSuccess && G_band) e = s.downward();
    if (e == cudaSuccess && G_1N) e = s.first_row((double2*)G_1N, (int64_t)p.b[0] * p.b[N - 1]);
  }
  if (e != cudaSuccess) { g_last_cuda = e; return NEGF_ERR_CUDA; }
  return NEGF_OK;
}
