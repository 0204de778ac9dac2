// Plan state of libnegf.so (one TU: included by negf_capi.cu only): the
// graph key of a call, the plan with its workspace layout, streams, events
// and profiling records, and the error helpers of the schedule code.
#pragma once

#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/negf.h"
#include "negf_common.cuh"
#include "negf_kernels.h"

using negf::ZGemm;

namespace {

struct CallKey {
  const void* p[12];
  int64_t stride;
  int kind;
  bool operator==(const CallKey& o) const {
    return kind == o.kind && stride == o.stride && std::memcmp(p, o.p, sizeof(p)) == 0;
  }
};

}  // namespace

// A per-energy workspace region of a DDRGF plan: offset (in units of one
// energy's elements times the chunk) and per-energy size; region r of energy
// e of the chunk lives at DDW + r.off * chunk + e * r.sz (one contiguous slab
// per region, so a batched launch over energies touches one slab).
struct DDReg { int64_t off = 0, sz = 0; };

// w-layer groups of one DDRGF sub-domain (step 1: fused sweeps of the closed
// sub-domain).  first / nl / sz: first layer, layers and elements of each
// group; hd / hu / hl: offsets of the energy-independent fused blocks
// H_{I,I}, H_{I,I+1}, H_{I+1,I}; t / x / y: per-energy regions of the
// right-connected sweep (t_I, X_I = t_I M_{I,I-1}, Y_I = M_{I-1,I} t_I).
struct DDGroups {
  std::vector<int> first, nl, sz;
  std::vector<int64_t> hd, hu, hl;
  std::vector<DDReg> t, x, y;
};

// One level of the DDRGF interface: a block tridiagonal chain of n nodes
// (the separators of the level above) with per-energy diagonal blocks D,
// couplings U (node k to k + 1) and L (k + 1 to k), whose left / right
// self-energies LL / RR every node needs.  A level that recurses is cut into
// np pairs: a group of nodes [f[J], l[J]] then the separator node l[J] + 1.
struct DDChain {
  int n = 0;
  std::vector<int> sz;                        // node sizes (elements)
  std::vector<DDReg> D, U, L, LL, RR;         // U / L: n - 1 entries
  int np = 0, child = -1;                     // pairs, index of the next level (-1: sequential sweeps)
  std::vector<int> f, l;                      // node range of each pair's group
  std::vector<DDReg> t, X, Y;                 // closed right sweep per node: t, t L_{k-1}, U_{k-1} t
  std::vector<DDReg> row, col;                // per pair: rings of the first row / column (2 slots)
  std::vector<DDReg> xll, s1, s2;             // per pair: X_LL, two node-sized temporaries
  std::vector<DDReg> cL, cR;                  // per separator node of a recursing level: group contributions
  std::vector<DDReg> tmp;                     // per node: a sweep temporary
};

struct negf_plan_s {
  int N = 0, w = 1, nE = 0, n_domains = 1, precision = 0, refine = 0, outputs = 0, ckpt = 0, bits = 0;
  long long wait_limit = -1;       // tensor-core MMA-completion wait polls (< 0: the kernel's default)
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
  // Keldysh on a block n-diagonal plan (w >= 2): a block tridiagonal
  // sub-plan on the fused chain (super-layers of w layers) runs negf_lesser
  // for fz_nE energies at a time; the band of H and the results move
  // between the two packings by block copies (fz_map: 7 int64 per original
  // band block), the lead terms are padded into the end super-blocks
  negf_plan_s* fz = nullptr;
  int fz_nE = 0, fz_nblk = 0, fz_rl = 0;       // energies per sub-call, blocks, layer N's offset in its super-block
  int64_t fz_elems = 0, fz_pad0 = 0, fz_padN = 0;   // fused band elements; end super-block sizes^2
  int64_t* fz_map = nullptr;                   // device map
  char* fz_buf = nullptr;                      // device buffers of the sub-calls
  double2 *fz_H = nullptr, *fz_E = nullptr, *fz_sL = nullptr, *fz_sR = nullptr, *fz_lL = nullptr, *fz_lR = nullptr,
          *fz_ld = nullptr, *fz_Gb = nullptr, *fz_Gl = nullptr;
  int32_t* fz_info = nullptr;
  negf_plan_s* fzg = nullptr;                  // the adjoint's sub-plan (every energy at once)
  char* fzg_buf = nullptr;
  double2 *fzg_H = nullptr, *fzg_dH = nullptr, *fzg_sL = nullptr, *fzg_sR = nullptr, *fzg_dL = nullptr,
          *fzg_dR = nullptr;
  int32_t* fzg_info = nullptr;
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
  // right separator D1_j = [dom_l[j] + 1, dom_l[j] + w].  F_j / L_j: the first
  // / last w layers of D2_j; P_j: the separator as one super-block.
  std::vector<int> dom_f, dom_l, Fsz, Lsz, Psz;
  std::vector<int> dom_of;                       // layer -> domain (-1: separator)
  std::vector<int> sep_of;                       // layer -> separator (-1: domain)
  std::vector<int> off_in;                       // layer offset inside F or the separator super-block
  int Pmax = 0, FLmax = 0, Bmax = 0;
  using Reg = DDReg;
  std::vector<DDGroups> grR, grL;               // step-1 groups (fused sweeps) per domain
  std::vector<int> lvl;                          // pair counts of the recursive interface levels
  std::vector<DDChain> chains;                   // interface levels: [0] the separators' chain
  std::vector<Reg> r_xll, r_xfl, r_xlf, r_lsS, r_lsG, r_lsY, r_row, r_col;   // per domain, step 1
  std::vector<Reg> r_wr, r_vr, r_sr, r_wl, r_vl, r_sl, r_tmp;                // per domain, step 4
  std::vector<Reg> r_A, r_cL, r_cR, r_base, r_LL, r_RR, r_gLs, r_gRin, r_gRs, r_Gpp, r_Tu, r_Tl;  // per separator
  Reg r_g1, r_g1t;
  int64_t dd_e = 0, hf_e = 0;
  std::vector<int64_t> mfp_off, mpf_off, mlq_off, mql_off;   // M super-blocks (offsets in Hf)
  double2* DDW = nullptr;       // per-energy DDRGF regions
  double2* Hf = nullptr;        // energy-independent fused H blocks and M super-blocks
  double2* band_ws = nullptr;   // band of one chunk when the caller keeps no band output

  // independent energy groups run on forked streams (graph branches)
  int groups = 1;
  int tc_cols = 512;   // tensor-core products: most TMEM columns per CTA (negf_autotune)
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;   // [0] fork, [1..] joins
  std::vector<cudaEvent_t> stagger;   // group g -> g + 1 start dependency
  // negf_solve_host with page-locked host outputs: each energy group copies
  // its band back in layer pieces on its own copy stream as the downward pass
  // completes them (created at the first such call)
  std::vector<cudaStream_t> cstream;
  std::vector<cudaEvent_t> cready, cdone;
  // DDRGF: the sub-domains of one energy group run concurrently, domain j of
  // group g on dstream[g * n_domains + j] (j = 0 on the group's own stream)
  std::vector<cudaStream_t> dstream;
  std::vector<cudaEvent_t> dfork, djoin;

  // optional per-launch timing (negf_profile_enable)
  bool profiling = false;
  struct Rec { int kind; double flops, issued; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  double prof_ms[NEGF_PROF_KINDS] = {0};
  double prof_flops[NEGF_PROF_KINDS] = {0};
  double prof_issued[NEGF_PROF_KINDS] = {0};
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

}  // namespace
