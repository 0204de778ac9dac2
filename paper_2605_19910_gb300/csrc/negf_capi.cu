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
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/negf.h"
#include "negf_common.cuh"
#include "negf_kernels.h"

#include "negf_plan.cuh"
#include "negf_sweep.cuh"
#include "negf_ddrgf.cuh"

using negf::ZGemm;

namespace {

// A per-energy self-energy stride must keep the energies' lead blocks apart
// (0 broadcasts one block to every energy): 0, or at least the larger lead
// block b_1^2, b_N^2.
bool bad_sigma_stride_sizes(int b_first, int b_last, int64_t stride) {
  if (stride < 0) return true;
  if (stride == 0) return false;
  return stride < std::max(sq(b_first), sq(b_last));
}
bool bad_sigma_stride(const negf_plan_s* p, int64_t stride) {
  return bad_sigma_stride_sizes(p->b[0], p->b[p->N - 1], stride);
}

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
  if (d->n_levels < 0 || (d->n_levels > 0 && !d->level_domains)) return NEGF_ERR_ARG;
  for (int k = 0; k < d->n_levels; ++k)
    if (d->level_domains[k] < 1) return NEGF_ERR_ARG;
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

int32_t negf_plan_levels(const negf_plan_t* p, int32_t* level_domains, int32_t cap) {
  if (!p) return -1;
  const int n = (int)p->lvl.size();
  for (int k = 0; k < n && k < cap && level_domains; ++k) level_domains[k] = p->lvl[k];
  return n;
}

}  // extern "C"

namespace {

// Eq. cost_model_RGF in units of one block GEMM with explicit inverses: the
// paper's LU is the inversion (ratio r_inv to a GEMM) and each GETRS is a
// GEMM with the inverse (r_GETRS = 1):
//   r_RGF(l) = l (4 + r_LU + 3 r_GETRS) - (4 + 2 r_GETRS).
double model_rgf(double l, double r_inv) { return l * (7.0 + r_inv) - 6.0; }
// r_RGF^extra(s2): the paper's values for s2 <= 4; beyond, the first and last
// rows and columns of the sub-domain inverse by chains of one GEMM per layer.
double model_extra(int s2) { return s2 <= 2 ? 0.0 : (s2 == 3 ? 2.0 : (s2 == 4 ? 6.0 : 4.0 * (s2 - 1))); }

struct ModelChoice {
  double cost = 1e300;
  std::vector<int> s2;    // per level
};

// Cost of DDRGF from level k on with l layers (nodes) of relative block cube
// scale `cube`, given the s2 candidates; returns the best and its s2 sequence.
void model_levels(double l, int s1, double cube, double r_inv, double nE, double slots, int depth, int max_levels,
                  const std::vector<int>& s2c, ModelChoice& best, std::vector<int>& seq) {
  // Concurrent tasks are graph branches of latency-bound launches.  Measured
  // on GB300 (1024 x 64 chain, one energy, FP64): 16 and 32 pairs take 234
  // and 217 ms, 113 pairs 482 ms, although every pair's step holds only a few
  // CTAs, so about 16 branches progress at once, not the ~128 concurrent
  // kernels the hardware admits: n_threads of the paper's model = 16.
  auto wave = [&](double tasks) { return std::max(std::max(1.0, tasks * nE / slots), tasks / 16.0); };
  // this level solved by RGF
  {
    const double c = wave(1.0) * model_rgf(l, r_inv) * cube;
    if (c < best.cost && depth > 0) { best.cost = c; best.s2 = seq; }
  }
  if (depth >= max_levels) return;
  for (int s2 : s2c) {
    if (s2 + s1 > l / 2) continue;                    // at least two pairs
    // pairs that each hold at least s2 + s1 layers (the paper rounds up; a
    // pair here must hold its whole group and separator)
    const double nt = std::floor(l / (double)(s2 + s1));
    if (nt > 128.0) continue;                          // one graph branch per pair, at most ~128 at once
    const double lvl = wave(nt) * cube *
                       (model_rgf(s2, r_inv) + model_extra(s2) + 4.0 * s2 + 4.0 + (4.0 * s2 + 4.0) +
                        (4.0 * (s2 - 1) + 2.0 * s2));
    // the next level: l_S = n_tasks s1 layers of super-blocks s1 times larger
    ModelChoice sub;
    std::vector<int> seq2 = seq;
    seq2.push_back(s2);
    const double cube2 = cube * (double)s1 * s1 * s1;
    model_levels(nt * s1, 1, cube2, r_inv, nE, slots, depth + 1, max_levels, {1, 2, 3, 4}, sub, seq2);
    if (lvl + sub.cost < best.cost) { best.cost = lvl + sub.cost; best.s2 = sub.s2; }
  }
}

}  // namespace

extern "C" {

// The paper's DDRGF cost model (Eq. cost_model_DDRGF with Eq. cost_model_RGF)
// evaluated for the GPU: see include/negf.h.
int32_t negf_ddrgf_model(int32_t n_blocks, const int32_t* block_sizes, int32_t band_n, int32_t n_energies,
                         int32_t sm_count, double r_inv, int32_t max_levels, int32_t* level_domains,
                         int32_t* n_levels, double* cost_rgf, double* cost_ddrgf) {
  if (n_levels) *n_levels = 0;
  if (n_blocks < 1 || !block_sizes || band_n < 3 || n_energies < 1 || sm_count < 1 || !(r_inv > 0.0)) return 1;
  const int w = (band_n - 1) / 2;
  int bmax = 1;
  for (int i = 0; i < n_blocks; ++i) bmax = std::max(bmax, (int)block_sizes[i]);
  const double per_cta = (double)bmax * (bmax + 1) * 16.0 + 1024.0;
  const double slots = bmax <= 119 ? (double)sm_count * std::min(5.0, std::max(1.0, std::floor(233472.0 / per_cta)))
                                   : std::max(1.0, std::floor(sm_count / 2.0));
  const double nE = n_energies;
  const double rgf = std::max(1.0, nE / slots) * model_rgf(n_blocks, r_inv);
  if (cost_rgf) *cost_rgf = rgf;
  ModelChoice best;
  best.cost = rgf;
  std::vector<int> s2c, seq;
  for (int m : {2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128}) s2c.push_back(m * w);
  model_levels(n_blocks, w, 1.0, r_inv, nE, slots, 0, std::max(1, (int)max_levels + 1), s2c, best, seq);
  if (cost_ddrgf) *cost_ddrgf = best.cost;
  if (best.s2.empty()) return 1;                      // plain RGF
  // level 1: pairs of s2 + w layers; deeper levels: pairs of s2 + 1 nodes
  double l = n_blocks;
  int nd = 1;
  for (size_t k = 0; k < best.s2.size(); ++k) {
    const int s1 = k == 0 ? w : 1;
    const int pairs = (int)std::floor(l / (double)(best.s2[k] + s1));
    if (k == 0) nd = pairs;
    else if (level_domains && (int)k - 1 < max_levels) level_domains[k - 1] = pairs;
    l = pairs;
  }
  if (n_levels) *n_levels = (int)best.s2.size() - 1;
  return nd;
}

}  // extern "C"

namespace {
std::mutex g_ratio_mu;
std::map<std::tuple<int, int, int>, double> g_ratio_cache;   // (device, b, precision) -> r_inv
}  // namespace

extern "C" {

negf_status negf_measure_r_inv(int32_t b, int32_t batch, int32_t precision, double* r_inv, void* cuda_stream) {
  if (b < 1 || b > NEGF_MAX_BLOCK || batch < 1 || !r_inv || (precision != NEGF_FP64 && precision != NEGF_MIXED))
    return NEGF_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NEGF_ERR_CUDA;
  cudaError_t e = negf::kernels_init();
  if (e != cudaSuccess) return cuda_status(e);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t elems = (size_t)batch * b * b;
  double2 *A = nullptr, *B = nullptr, *Cm = nullptr;
  int32_t* info = nullptr;
  int* err = nullptr;
  e = cudaMalloc((void**)&A, elems * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&B, elems * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&Cm, elems * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&info, sizeof(int32_t) * batch + sizeof(int));
  if (e != cudaSuccess) {
    cudaFree(A); cudaFree(B); cudaFree(Cm); cudaFree(info);
    g_last_cuda = e; cudaGetLastError();
    return NEGF_ERR_NOMEM;
  }
  err = reinterpret_cast<int*>(info + batch);
  cudaEvent_t a = nullptr, z = nullptr;
  float t_inv = 0.f, t_mm = 0.f;
  e = cudaMemsetAsync(info, 0, sizeof(int32_t) * batch + sizeof(int), st);
  if (e == cudaSuccess) e = negf::set_identity(A, (int64_t)b * b, b, batch, st);   // regular operands
  if (e == cudaSuccess) e = negf::set_identity(B, (int64_t)b * b, b, batch, st);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&z);
  ZGemm g;
  g.m = b; g.n = b; g.k = b;
  g.A = A; g.sA = (int64_t)b * b; g.lda = b;
  g.B = B; g.sB = (int64_t)b * b; g.ldb = b;
  g.C = Cm; g.sC = (int64_t)b * b; g.ldc = b;
  g.errword = err;
  g.bits = NEGF_DEFAULT_PRODUCT_BITS;
  g.batch = batch;
  auto prod = [&]() { return precision == NEGF_MIXED ? negf::zgemm_tc(g, st) : negf::zgemm_f64(g, st); };
  const int reps = 10;
  for (int r = 0; r < 3 && e == cudaSuccess; ++r) {   // warm-up
    e = negf::zinv_f64(A, (int64_t)b * b, Cm, (int64_t)b * b, b, batch, info, 1, err, st);
    if (e == cudaSuccess) e = prod();
  }
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  for (int r = 0; r < reps && e == cudaSuccess; ++r)
    e = negf::zinv_f64(A, (int64_t)b * b, Cm, (int64_t)b * b, b, batch, info, 1, err, st);
  if (e == cudaSuccess) e = cudaEventRecord(z, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(z);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t_inv, a, z);
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = prod();
  if (e == cudaSuccess) e = cudaEventRecord(z, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(z);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t_mm, a, z);
  if (a) cudaEventDestroy(a);
  if (z) cudaEventDestroy(z);
  cudaFree(A); cudaFree(B); cudaFree(Cm); cudaFree(info);
  if (e != cudaSuccess) return cuda_status(e);
  *r_inv = t_mm > 0.f ? (double)t_inv / (double)t_mm : 1.0;
  std::lock_guard<std::mutex> lk(g_ratio_mu);
  g_ratio_cache[std::make_tuple(dev, (int)b, (int)precision)] = *r_inv;
  return NEGF_OK;
}

}  // extern "C"

namespace {

// Keldysh and the adjoint on a block n-diagonal plan run on its fused
// block tridiagonal chain (Sec. 2.3, block fusing: super-layer J holds layers
// [J w, (J + 1) w), the last one possibly fewer): a sub-plan on the
// super-blocks, the block map between the two band packings and the device
// buffers of the sub-calls.  The adjoint of a DDRGF plan runs the same way on
// a plain RGF sub-plan of its chain (w = 1: the map is the identity layout).  The Keldysh sub-calls take fz_nE energies at a
// time so that the fused outputs stay within about 8 GiB; the adjoint's take
// every energy (its fused outputs are one band and the leads' gradients).
negf_status fused_setup(negf_plan_s* p, const negf_desc* d) {
  const int N = p->N, w = p->w, Nf = (N + w - 1) / w;
  std::vector<int32_t> fs(Nf, 0);
  std::vector<int> start(N + 1, 0), fstart(Nf + 1, 0);
  for (int i = 0; i < N; ++i) { fs[i / w] += p->b[i]; start[i + 1] = start[i] + p->b[i]; }
  for (int J = 0; J < Nf; ++J) fstart[J + 1] = fstart[J] + fs[J];
  // fused band offsets (block tridiagonal packing: diagonals -1, 0, +1, layers inner)
  std::vector<int64_t> foff((size_t)3 * Nf, -1);
  int64_t fe = 0;
  for (int dd = -1; dd <= 1; ++dd)
    for (int J = 0; J < Nf; ++J)
      if (J + dd >= 0 && J + dd < Nf) { foff[(size_t)(dd + 1) * Nf + J] = fe; fe += (int64_t)fs[J] * fs[J + dd]; }
  std::vector<int64_t> map;
  for (int dd = -w; dd <= w; ++dd)
    for (int a = 0; a < N; ++a) {
      const int b = a + dd;
      if (b < 0 || b >= N) continue;
      const int J = a / w, K = b / w;
      map.push_back(p->band_off[(size_t)(dd + w) * N + a]);
      map.push_back(p->b[a]);
      map.push_back(p->b[b]);
      map.push_back(foff[(size_t)(K - J + 1) * Nf + J]);
      map.push_back(fs[K]);
      map.push_back(start[a] - fstart[J]);
      map.push_back(start[b] - fstart[K]);
    }
  p->fz_nblk = (int)(map.size() / 7);
  p->fz_elems = fe;
  p->fz_rl = start[N - 1] - fstart[Nf - 1];
  p->fz_pad0 = sq(fs[0]);
  p->fz_padN = sq(fs[Nf - 1]);
  const int64_t pad = std::max(p->fz_pad0, p->fz_padN);
  cudaError_t e = cudaMalloc((void**)&p->fz_map, map.size() * sizeof(int64_t));
  if (e != cudaSuccess) { g_last_cuda = e; cudaGetLastError(); return NEGF_ERR_NOMEM; }
  e = cudaMemcpy(p->fz_map, map.data(), map.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_status(e);
  negf_desc sd = *d;
  sd.n_blocks = Nf;
  sd.block_sizes = fs.data();
  sd.band_n = 3;
  sd.product_bits = p->bits;
  sd.refine_steps = 0;
  sd.n_domains = 1;
  sd.domain_first_block = nullptr;
  sd.n_levels = 0;
  sd.level_domains = nullptr;
  if ((d->outputs & NEGF_OUT_LESSER) && w > 1) {
    const double per_e = 2.0 * (double)fe * sizeof(double2);
    p->fz_nE = (int)std::max(1.0, std::min((double)p->nE, std::floor(8.0 * (1ull << 30) / per_e)));
    negf_desc ld = sd;
    ld.n_energies = p->fz_nE;
    ld.outputs = NEGF_OUT_BAND | NEGF_OUT_LESSER;
    ld.checkpoint_every = 0;
    negf_status st = negf_plan(&p->fz, &ld, p->stream);
    if (st != NEGF_OK) return st;
    const int64_t nEs = p->fz_nE;
    const size_t elems = (size_t)(fe + nEs + 4 * nEs * pad + nEs + 2 * nEs * fe);
    e = cudaMalloc((void**)&p->fz_buf, elems * sizeof(double2) + (size_t)nEs * sizeof(int32_t));
    if (e != cudaSuccess) { g_last_cuda = e; cudaGetLastError(); return NEGF_ERR_NOMEM; }
    double2* q = reinterpret_cast<double2*>(p->fz_buf);
    p->fz_H = q; q += fe;
    p->fz_E = q; q += nEs;
    p->fz_sL = q; q += nEs * pad;
    p->fz_sR = q; q += nEs * pad;
    p->fz_lL = q; q += nEs * pad;
    p->fz_lR = q; q += nEs * pad;
    p->fz_ld = q; q += nEs;
    p->fz_Gb = q; q += nEs * fe;
    p->fz_Gl = q; q += nEs * fe;
    p->fz_info = reinterpret_cast<int32_t*>(q);
  }
  if (d->outputs & NEGF_OUT_GRAD) {
    negf_desc gd = sd;
    gd.outputs = NEGF_OUT_GRAD;   // checkpoint_every passes through
    negf_status st = negf_plan(&p->fzg, &gd, p->stream);
    if (st != NEGF_OK) return st;
    const int64_t nE = p->nE;
    const size_t elems = (size_t)(2 * fe + 4 * nE * pad);
    e = cudaMalloc((void**)&p->fzg_buf, elems * sizeof(double2) + (size_t)nE * sizeof(int32_t));
    if (e != cudaSuccess) { g_last_cuda = e; cudaGetLastError(); return NEGF_ERR_NOMEM; }
    double2* q = reinterpret_cast<double2*>(p->fzg_buf);
    p->fzg_H = q; q += fe;
    p->fzg_dH = q; q += fe;
    p->fzg_sL = q; q += nE * pad;
    p->fzg_sR = q; q += nE * pad;
    p->fzg_dL = q; q += nE * pad;
    p->fzg_dR = q; q += nE * pad;
    p->fzg_info = reinterpret_cast<int32_t*>(q);
  }
  return NEGF_OK;
}

// b x b lead matrices padded into zeroed fsz x fsz blocks at (at, at): with
// a per-energy stride, nEs blocks at dstride (the chunk's n energies, then
// the last one repeated for a short last chunk); shared (stride 0): one.
cudaError_t fused_pad(const double2* src, int64_t stride, int b, double2* dst, int64_t dstride, int fsz, int at,
                      int n, int nEs, cudaStream_t st) {
  const int cnt = stride ? nEs : 1;
  const int64_t ds = stride ? dstride : (int64_t)fsz * fsz;
  NEGF_TRY(cudaMemsetAsync(dst, 0, sizeof(double2) * (size_t)(cnt * ds), st));
  double2* d0 = dst + (int64_t)at * fsz + at;
  if (!stride) return negf::copy2d(src, 0, b, d0, ds, fsz, b, b, 1.0, 0, 1, st);
  NEGF_TRY(negf::copy2d(src, stride, b, d0, ds, fsz, b, b, 1.0, 0, n, st));
  if (n < nEs) NEGF_TRY(negf::copy2d(src + (int64_t)(n - 1) * stride, 0, b, d0 + (int64_t)n * ds, ds, fsz, b, b, 1.0, 0,
                                     nEs - n, st));
  return cudaSuccess;
}

// negf_lesser of a block n-diagonal plan through its fused chain.
negf_status fused_lesser(negf_plan_s* p, const double2* H, const double2* sigma_L, const double2* sigma_R,
                         int64_t sigma_E_stride, const double2* E, const double2* sigma_less_L,
                         const double2* sigma_less_R, int64_t sless_stride, const double2* less_diag,
                         double2* G_band, double2* G_less, int32_t* info) {
  negf_plan_s* f = p->fz;
  cudaStream_t st = p->stream;
  const int N = p->N, Nf = f->N, nEs = p->fz_nE;
  const int b0 = p->b[0], bN = p->b[N - 1], fs0 = f->b[0], fsN = f->b[Nf - 1];
  NEGF_TRY_STATUS(cudaMemsetAsync(p->fz_H, 0, sizeof(double2) * (size_t)p->fz_elems, st));
  NEGF_TRY_STATUS(negf::band_remap(H, 0, p->fz_H, 0, p->fz_map, p->fz_nblk, 1, 0, st));
  for (int e0 = 0; e0 < p->nE; e0 += nEs) {
    const int n = std::min(nEs, p->nE - e0);
    // energies of this sub-call; a short last call repeats its last energy
    NEGF_TRY_STATUS(cudaMemcpyAsync(p->fz_E, E + e0, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st));
    if (n < nEs) NEGF_TRY_STATUS(negf::copy2d(E + e0 + n - 1, 0, 1, p->fz_E + n, 1, 1, 1, 1, 1.0, 0, nEs - n, st));
    // padded leads: per-energy ones at the larger end block's size squared
    // (one layout for both ends), shared ones as one block (stride 0)
    const int64_t pad = std::max(p->fz_pad0, p->fz_padN);
    const int64_t ps = sigma_E_stride ? pad : 0, ls = sless_stride ? pad : 0;
    const double2 *pL = nullptr, *pR = nullptr, *lL = nullptr, *lR = nullptr, *ld = nullptr;
    if (sigma_L) {
      NEGF_TRY_STATUS(fused_pad(sigma_L + e0 * sigma_E_stride, sigma_E_stride, b0, p->fz_sL, pad, fs0, 0, n, nEs, st));
      pL = p->fz_sL;
    }
    if (sigma_R) {
      NEGF_TRY_STATUS(fused_pad(sigma_R + e0 * sigma_E_stride, sigma_E_stride, bN, p->fz_sR, pad, fsN, p->fz_rl, n,
                                nEs, st));
      pR = p->fz_sR;
    }
    if (sigma_less_L) {
      NEGF_TRY_STATUS(fused_pad(sigma_less_L + e0 * sless_stride, sless_stride, b0, p->fz_lL, pad, fs0, 0, n, nEs, st));
      lL = p->fz_lL;
    }
    if (sigma_less_R) {
      NEGF_TRY_STATUS(fused_pad(sigma_less_R + e0 * sless_stride, sless_stride, bN, p->fz_lR, pad, fsN, p->fz_rl, n,
                                nEs, st));
      lR = p->fz_lR;
    }
    if (less_diag) {
      NEGF_TRY_STATUS(cudaMemsetAsync(p->fz_ld, 0, sizeof(double2) * nEs, st));
      NEGF_TRY_STATUS(cudaMemcpyAsync(p->fz_ld, less_diag + e0, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st));
      ld = p->fz_ld;
    }
    auto c = [](const double2* x) { return reinterpret_cast<const negf_c128*>(x); };
    negf_status s = negf_lesser(f, c(p->fz_H), c(pL), c(pR), ps, c(p->fz_E), c(lL), c(lR), ls, c(ld),
                                reinterpret_cast<negf_c128*>(p->fz_Gb), reinterpret_cast<negf_c128*>(p->fz_Gl),
                                p->fz_info);
    if (s != NEGF_OK) return s;
    NEGF_TRY_STATUS(negf::band_remap(p->fz_Gb, p->fz_elems, G_band + (int64_t)e0 * p->band_elems, p->band_elems,
                                     p->fz_map, p->fz_nblk, n, 1, st));
    NEGF_TRY_STATUS(negf::band_remap(p->fz_Gl, p->fz_elems, G_less + (int64_t)e0 * p->band_elems, p->band_elems,
                                     p->fz_map, p->fz_nblk, n, 1, st));
    NEGF_TRY_STATUS(negf::fold_fused_status(info + e0, p->fz_info, n, p->w, p->d_err, f->d_err, st));
  }
  return NEGF_OK;
}

// negf_grad_strided of a block n-diagonal plan through its fused chain: the
// fused H is the original band laid out on super-blocks (zeros elsewhere), so
// each original block's gradient is its sub-block of the super-block's
// gradient, and the leads' gradients are the sub-blocks where the leads
// were padded in.
negf_status fused_grad(negf_plan_s* p, const double2* H, const double2* sigma_L, const double2* sigma_R,
                       int64_t sigma_E_stride, const double2* E, const double* dL_dT, double* T, double2* dH,
                       double2* dSigma_L, int64_t dL_stride, double2* dSigma_R, int64_t dR_stride, int32_t* info) {
  negf_plan_s* f = p->fzg;
  cudaStream_t st = p->stream;
  const int N = p->N, Nf = f->N, nE = p->nE;
  const int b0 = p->b[0], bN = p->b[N - 1], fs0 = f->b[0], fsN = f->b[Nf - 1];
  const int64_t pad = std::max(p->fz_pad0, p->fz_padN);
  NEGF_TRY_STATUS(cudaMemsetAsync(p->fzg_H, 0, sizeof(double2) * (size_t)p->fz_elems, st));
  NEGF_TRY_STATUS(negf::band_remap(H, 0, p->fzg_H, 0, p->fz_map, p->fz_nblk, 1, 0, st));
  NEGF_TRY_STATUS(fused_pad(sigma_L, sigma_E_stride, b0, p->fzg_sL, pad, fs0, 0, nE, nE, st));
  NEGF_TRY_STATUS(fused_pad(sigma_R, sigma_E_stride, bN, p->fzg_sR, pad, fsN, p->fz_rl, nE, nE, st));
  const int64_t ps = sigma_E_stride ? pad : 0, pls = dL_stride ? pad : 0, prs = dR_stride ? pad : 0;
  auto c = [](const double2* x) { return reinterpret_cast<const negf_c128*>(x); };
  auto m = [](double2* x) { return reinterpret_cast<negf_c128*>(x); };
  negf_status s = negf_grad_strided(f, c(p->fzg_H), c(p->fzg_sL), c(p->fzg_sR), ps, c(E), dL_dT, T, m(p->fzg_dH),
                                    dSigma_L ? m(p->fzg_dL) : nullptr, pls, dSigma_R ? m(p->fzg_dR) : nullptr, prs,
                                    p->fzg_info);
  if (s != NEGF_OK) return s;
  NEGF_TRY_STATUS(negf::band_remap(p->fzg_dH, 0, dH, 0, p->fz_map, p->fz_nblk, 1, 1, st));
  if (dSigma_L)
    NEGF_TRY_STATUS(negf::copy2d(p->fzg_dL, pls, fs0, dSigma_L, dL_stride, b0, b0, b0, 1.0, 0, dL_stride ? nE : 1, st));
  if (dSigma_R)
    NEGF_TRY_STATUS(negf::copy2d(p->fzg_dR + (int64_t)p->fz_rl * fsN + p->fz_rl, prs, fsN, dSigma_R, dR_stride, bN,
                                 bN, bN, 1.0, 0, dR_stride ? nE : 1, st));
  NEGF_TRY_STATUS(negf::fold_fused_status(info, p->fzg_info, nE, p->w, p->d_err, f->d_err, st));
  return NEGF_OK;
}

}  // namespace

extern "C" {

negf_status negf_plan(negf_plan_t** out, const negf_desc* din, void* cuda_stream) {
  if (!out) return NEGF_ERR_ARG;
  *out = nullptr;
  negf_status v = validate(din);
  if (v != NEGF_OK) return v;
  negf_desc dd_auto = *din;
  const negf_desc* d = &dd_auto;
  std::vector<int32_t> auto_levels(8, 0);
  if (dd_auto.n_domains == 0) {
    // the paper's cost model (Eq. cost_model_DDRGF) with this GPU's measured
    // ratio of a batched block inversion to a batched block product picks
    // plain RGF or DDRGF, its pair count and the interface levels
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      sms = 152;
    }
    if (din->outputs & NEGF_OUT_GRAD) {
      dd_auto.n_domains = 1;
    } else {
      int bmax = 1;
      for (int i = 0; i < din->n_blocks; ++i) bmax = std::max(bmax, (int)din->block_sizes[i]);
      double r = 0.0;
      {
        std::lock_guard<std::mutex> lk(g_ratio_mu);
        auto it = g_ratio_cache.find(std::make_tuple(dev, bmax, (int)din->precision));
        if (it != g_ratio_cache.end()) r = it->second;
      }
      if (r <= 0.0) {
        const negf_status ms = negf_measure_r_inv(bmax, std::min(din->n_energies, 512), din->precision, &r, nullptr);
        if (ms != NEGF_OK) return ms;
      }
      int32_t nl = 0;
      dd_auto.n_domains = negf_ddrgf_model(din->n_blocks, din->block_sizes, din->band_n, din->n_energies, sms, r,
                                           (int32_t)auto_levels.size(), auto_levels.data(), &nl, nullptr, nullptr);
      dd_auto.n_levels = dd_auto.n_domains > 1 ? nl : 0;
      dd_auto.level_domains = dd_auto.n_levels ? auto_levels.data() : nullptr;
    }
  }
  const int w = (d->band_n - 1) / 2;
  if (d->precision == NEGF_MIXED && !negf::zgemm_tc_available()) return NEGF_ERR_UNSUPPORTED;
  if ((d->outputs & NEGF_OUT_LESSER) && (d->n_domains > 1 || (d->checkpoint_every > 0 && (d->outputs & NEGF_OUT_GRAD))))
    return NEGF_ERR_UNSUPPORTED;
  if ((d->outputs & (NEGF_OUT_LESSER | NEGF_OUT_GRAD)) && w > 1)   // the fused chain's super-blocks must invert
    for (int i = 0; i < d->n_blocks; i += w) {
      int64_t sz = 0;
      for (int j = i; j < std::min(d->n_blocks, i + w); ++j) sz += d->block_sizes[j];
      if (sz > negf::zinv_max_block()) return NEGF_ERR_UNSUPPORTED;
    }
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
  // mixed plans default to NEGF_DEFAULT_PRODUCT_BITS (negf_tune_precision
  // can narrow it on the caller's inputs)
  p->bits = d->product_bits ? d->product_bits : (d->precision == NEGF_MIXED ? NEGF_DEFAULT_PRODUCT_BITS : 0);
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
      // every pair keeps at least 3w layers (a sub-domain of 2w, a separator of w)
      for (int j = 1; j < nd; ++j) first[j] = std::max(first[j], first[j - 1] + 3 * w);
      for (int j = nd - 1; j >= 1; --j) first[j] = std::min(first[j], (j + 1 < nd ? first[j + 1] : N) - 3 * w);
    }
    p->dom_f.resize(nd); p->dom_l.resize(nd);
    for (int j = 0; j < nd; ++j) {
      const int lo = first[j], hi = (j + 1 < nd) ? first[j + 1] : N;   // pair = [lo, hi)
      // a pair holds its sub-domain (at least 2w layers: disjoint first and
      // last w layers) and its separator of w layers
      if ((j == 0 && lo != 0) || hi - lo < 3 * w) { delete p; return NEGF_ERR_ARG; }
      p->dom_f[j] = lo;
      p->dom_l[j] = hi - w - 1;
    }
    p->lvl.assign(d->level_domains ? d->level_domains : nullptr,
                  d->level_domains ? d->level_domains + d->n_levels : nullptr);
    const int lay = dd_layout(p, negf::zinv_max_block());
    if (lay != 0) { delete p; return lay < 0 ? NEGF_ERR_ARG : NEGF_ERR_UNSUPPORTED; }
    dd_e = p->dd_e + p->band_elems;
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
  // block n-diagonal and DDRGF plans run the adjoint on a sub-plan (the
  // fused chain, or the same chain by plain RGF)
  const bool grad = (d->outputs & NEGF_OUT_GRAD) != 0 && w == 1 && p->n_domains == 1;
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
  int64_t ck_elems = 0;
  if (p->ck_k > 0) {
    p->p_elems = (int64_t)(p->ck_k + 1) * p->bmaxN;
    ck_elems = (int64_t)p->ck_nseg * (p->bmax2 + p->bmaxN);
  }
  // Gamma_L, Gamma_R, P, Q, G_1N, and two more b1 x bN temporaries (gradient)
  p->scr_elems = sq(b0) + sq(bN) + 5 * (int64_t)b0 * bN;

  const int64_t lesser_e = ((d->outputs & NEGF_OUT_LESSER) && w == 1) ? 2 * te : 0;
  const int64_t dh_e = grad ? p->bmax2 : 0;
  int64_t per_e = dh_e + lesser_e + te + xe + ye + (int64_t)(w + 1) * (w + 1) * p->s_slot * std::max(1, p->n_domains) +
                  (p->full_row ? re : (int64_t)(w + 1) * b0 * bmax) + 2 * p->p_elems + ck_elems +
                  p->scr_elems + dd_e;
  // chunk energies so that the workspace stays within a budget: 45% of the
  // device memory free at plan time, at least 24 GiB (the caller's outputs
  // need the rest)
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); free_b = 0; }
  double budget_bytes = std::max(24.0 * (1ull << 30), 0.45 * (double)free_b);
  if (const char* cap = getenv("NEGF_WORKSPACE_GB")) {   // caller's cap (energies are chunked to fit)
    const double gb = atof(cap);
    if (gb > 0.0) budget_bytes = gb * (double)(1ull << 30);
  }
  const int64_t budget_elems = (int64_t)(budget_bytes / (double)sizeof(double2));
  int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(p->nE, budget_elems / std::max<int64_t>(per_e, 1)));
  p->chunk = chunk;
  p->ws_bytes = (size_t)(per_e * chunk + p->hf_e) * sizeof(double2) + 256;
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
    p->DDW = q; q += p->dd_e * chunk;
    p->band_ws = q; q += p->band_elems * chunk;
    p->Hf = q; q += p->hf_e;
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
  if (((d->outputs & NEGF_OUT_LESSER) && w > 1) || ((d->outputs & NEGF_OUT_GRAD) && (w > 1 || p->n_domains > 1))) {
    const negf_status fs = fused_setup(p, d);
    if (fs != NEGF_OK) { negf_destroy(p); return fs; }
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
  for (auto c : p->cstream) cudaStreamDestroy(c);
  for (auto c : p->cready) cudaEventDestroy(c);
  for (auto c : p->cdone) cudaEventDestroy(c);
  cudaFree(p->ws);
  cudaFree(p->d_err);
  if (p->host_io) cudaFree(p->host_io);
  if (p->fz) negf_destroy(p->fz);
  if (p->fzg) negf_destroy(p->fzg);
  if (p->fz_map) cudaFree(p->fz_map);
  if (p->fz_buf) cudaFree(p->fz_buf);
  if (p->fzg_buf) cudaFree(p->fzg_buf);
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
  // a wait that gave up leaves the product unwritten: later pivots are
  // consequences, so the timeout is reported first
  if (word & negf::ERRBIT_TIMEOUT) return NEGF_ERR_TIMEOUT;
  if (word & negf::ERRBIT_NONFINITE) return NEGF_ERR_NONFINITE;
  if (word & negf::ERRBIT_SINGULAR) return NEGF_ERR_SINGULAR;
  return NEGF_OK;
}


}  // extern "C"

namespace {


enum CallKind { CALL_SOLVE = 1, CALL_TRANS = 2, CALL_GRAD = 3, CALL_SOLVE_HOST = 5 };

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

namespace {

// The schedule of negf_solve on device buffers.  With host_band / host_g1n
// (page-locked host memory, plain RGF plans) every energy group also copies
// its band back in layer pieces on its own copy stream as its downward pass
// completes them, and its G_1N after that; the copy streams join the plan's
// stream at the end.
cudaError_t solve_body(negf_plan_s* p, const negf_c128* H, const negf_c128* sigma_L, const negf_c128* sigma_R,
                       int64_t sigma_E_stride, const negf_c128* E, negf_c128* G_band, negf_c128* G_1N,
                       int32_t* info, negf_c128* host_band, negf_c128* host_g1n) {
  NEGF_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t) * p->nE, p->stream));
  const bool host = host_band || host_g1n;
  const int64_t s1 = (int64_t)p->b[0] * p->b[p->N - 1];
  for (int e0 = 0; e0 < p->nE; e0 += p->chunk) {
    Sweep base{p, p->stream, (const double2*)H, (const double2*)sigma_L, (const double2*)sigma_R,
               sigma_E_stride, (const double2*)E, (double2*)G_band, (double2*)G_1N, info,
               e0, std::min(p->chunk, p->nE - e0)};
    if (p->n_domains > 1) {
      if (!G_band) { base.Gband = p->band_ws; base.gb_e0 = e0; }
      if (e0 == 0) NEGF_TRY(DD(p, base).assemble_static());
      NEGF_TRY(for_groups(p, base, [&](Sweep& s) -> cudaError_t {
        return DD(p, s).run(true, G_1N ? (double2*)G_1N + (int64_t)s.e0 * s1 : nullptr, s1);
      }));
      continue;
    }
    NEGF_TRY(for_groups(p, base, [&](Sweep& s) -> cudaError_t {
      if (host) {
        s.host_band = (double2*)host_band;
        s.cst = p->cstream[s.grp];
        s.cready = p->cready[s.grp];
      }
      if (p->ck_k > 0) {
        NEGF_TRY(s.ck_forward((double2*)G_1N + (int64_t)s.e0 * s1, s1));
      } else {
        NEGF_TRY(s.upward(G_band != nullptr || (G_1N && p->refine)));
        if (G_band) NEGF_TRY(s.downward());
        if (G_1N && p->refine) {   // G_1N = first block of the last column, refined
          NEGF_TRY(s.last_column());
          NEGF_TRY(s.refine_g1n((double2*)G_1N + (int64_t)s.e0 * s1, s1));
        } else if (G_1N) {
          NEGF_TRY(s.first_row((double2*)G_1N + (int64_t)s.e0 * s1, s1));
        }
      }
      if (host_g1n) {
        NEGF_TRY(cudaEventRecord(s.cready, s.st));
        NEGF_TRY(cudaStreamWaitEvent(s.cst, s.cready, 0));
        NEGF_TRY(cudaMemcpyAsync(host_g1n + (int64_t)s.e0 * s1, G_1N + (int64_t)s.e0 * s1,
                                 (size_t)(s.ne * s1) * sizeof(negf_c128), cudaMemcpyDeviceToHost, s.cst));
      }
      return cudaSuccess;
    }));
  }
  if (host) {   // join every group's copy stream
    const int G = std::min(p->groups, p->chunk);
    for (int g = 0; g < G; ++g) {
      NEGF_TRY(cudaEventRecord(p->cdone[g], p->cstream[g]));
      NEGF_TRY(cudaStreamWaitEvent(p->stream, p->cdone[g], 0));
    }
  }
  return cudaSuccess;
}

}  // namespace

extern "C" {

negf_status negf_solve(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                       const negf_c128* sigma_R, int64_t sigma_E_stride, const negf_c128* E,
                       negf_c128* G_band, negf_c128* G_1N, int32_t* info) {
  if (!p || !H || !E || !info || bad_sigma_stride(p, sigma_E_stride)) return NEGF_ERR_ARG;
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
    return solve_body(p, H, sigma_L, sigma_R, sigma_E_stride, E, G_band, G_1N, info, nullptr, nullptr);
  });
}

negf_status negf_transmission(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                              const negf_c128* sigma_R, int64_t sigma_E_stride, const negf_c128* E,
                              double* T, int32_t* info) {
  if (!p || !H || !E || !info || !T || !sigma_L || !sigma_R || bad_sigma_stride(p, sigma_E_stride)) return NEGF_ERR_ARG;
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
        if (e0 == 0) NEGF_TRY(DD(p, base).assemble_static());
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
          NEGF_TRY(s.refine_g1n(g1n, s1));
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
  return negf_grad_strided(p, H, sigma_L, sigma_R, sigma_E_stride, E, dL_dT, T, dH, dSigma_L, sigma_E_stride,
                           dSigma_R, sigma_E_stride, info);
}

negf_status negf_grad_strided(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                              const negf_c128* sigma_R, int64_t sigma_E_stride, const negf_c128* E,
                              const double* dL_dT, double* T, negf_c128* dH, negf_c128* dSigma_L,
                              int64_t dSigma_L_stride, negf_c128* dSigma_R, int64_t dSigma_R_stride,
                              int32_t* info) {
  if (!p || !H || !E || !info || !dL_dT || !dH || !sigma_L || !sigma_R || bad_sigma_stride(p, sigma_E_stride))
    return NEGF_ERR_ARG;
  if (bad_sigma_stride(p, dSigma_L_stride) || bad_sigma_stride(p, dSigma_R_stride)) return NEGF_ERR_ARG;
  if (!(p->outputs & NEGF_OUT_GRAD)) return NEGF_ERR_ARG;
  if (p->w > 1 || p->n_domains > 1)
    return p->fzg ? fused_grad(p, (const double2*)H, (const double2*)sigma_L, (const double2*)sigma_R, sigma_E_stride,
                               (const double2*)E, dL_dT, T, (double2*)dH, (double2*)dSigma_L, dSigma_L_stride,
                               (double2*)dSigma_R, dSigma_R_stride, info)
                  : NEGF_ERR_UNSUPPORTED;
  CallKey key{};
  key.kind = CALL_GRAD;
  key.stride = sigma_E_stride;
  const void* ptrs[] = {H, sigma_L, sigma_R, E, dL_dT, T, dH, dSigma_L, dSigma_R, info,
                        (const void*)(intptr_t)dSigma_L_stride, (const void*)(intptr_t)dSigma_R_stride};
  std::memcpy(key.p, ptrs, sizeof(ptrs));
  // output stride of the gradient of Sigma_L (side 0) / Sigma_R (side 1): 0 sums over energies
  auto ostride = [&](int side) { return side == 0 ? dSigma_L_stride : dSigma_R_stride; };
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
        const int64_t os = ostride(side);
        if (!dS || os == 0) return cudaSuccess;
        const int bs = side == 0 ? b0 : bN;
        ZGemm h;
        h.m = bs; h.n = bs; h.k = bN;
        h.A = Ui; h.sA = sUi; h.lda = bs; h.opA = negf::OP_C;
        h.B = Li; h.sB = sLi; h.ldb = bN; h.opB = negf::OP_C;
        h.C = (double2*)dS + (int64_t)e0 * os; h.sC = os; h.ldc = bs;
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
        const int64_t os = ostride(side);
        if (os == 0) {   // per-energy products, then their weighted sum times -2i
          g.C = p->DH_ws; g.sC = p->bmax2; g.ldc = bs;
          NEGF_TRY(s.gemm64(g));
          NEGF_TRY(s.misc([&] {
            return negf::reduce_energies(p->DH_ws, p->bmax2, bs, ne, dL_dT + e0, (double2*)dS, bs, bs, bs,
                                         {0.0, -2.0}, first ? 0 : 1, 0, p->stream);
          }));
        } else {   // per energy, onto the M-path part written above
          double2* out = (double2*)dS + (int64_t)e0 * os;
          g.alpha = {0.0, -2.0};
          g.weight = dL_dT + e0;
          g.C = out; g.sC = os; g.ldc = bs;
          g.C1 = out; g.sC1 = os; g.ldc1 = bs; g.beta1 = {1.0, 0.0};
          NEGF_TRY(s.gemm64(g));
        }
      }
    }
    {   // summed outputs: add the M-path parts dH_00 / dH_NN once, after all chunks
      Sweep s{p, p->stream, nullptr, nullptr, nullptr, 0, nullptr, nullptr, nullptr, info, 0, 1};
      for (int side = 0; side < 2; ++side) {
        negf_c128* dS = side == 0 ? dSigma_L : dSigma_R;
        if (!dS || ostride(side) != 0) continue;
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
namespace {

bool host_pinned(const void* ptr) {
  if (!ptr) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeHost;
}

// Copy streams and events of negf_solve_host's overlapped copies.
cudaError_t ensure_copy_streams(negf_plan_s* p) {
  const int G = (int)p->side.size() + 1;
  while ((int)p->cstream.size() < G) {
    cudaStream_t c = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    NEGF_TRY(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
    p->cstream.push_back(c);
    NEGF_TRY(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
    p->cready.push_back(a);
    NEGF_TRY(cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
    p->cdone.push_back(b);
  }
  return cudaSuccess;
}

}  // namespace

// negf_solve from host memory to host memory: inputs copied to device
// buffers the plan owns, the captured solve, outputs copied back, all on the
// plan's stream; returns after the outputs are in host memory (with
// negf_sync's status).  With page-locked outputs on a plain RGF plan the
// band's copy back overlaps the solve (piecewise, per energy group).
negf_status negf_solve_host(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                            const negf_c128* sigma_R, int64_t sigma_E_stride, const negf_c128* E,
                            negf_c128* G_band, negf_c128* G_1N, int32_t* info) {
  if (!p || !H || !E || !info || bad_sigma_stride(p, sigma_E_stride) || (!G_band && !G_1N)) return NEGF_ERR_ARG;
  if (p->ck_k > 0 && G_band) return NEGF_ERR_UNSUPPORTED;
  const int64_t nE = p->nE, b0 = p->b[0], bN = p->b[p->N - 1];
  const int64_t nsig_L = sigma_E_stride ? (nE - 1) * sigma_E_stride + b0 * b0 : b0 * b0;
  const int64_t nsig_R = sigma_E_stride ? (nE - 1) * sigma_E_stride + bN * bN : bN * bN;
  auto al = [](int64_t elems) { return (size_t)((elems * (int64_t)sizeof(double2) + 255) / 256 * 256); };
  const size_t oH = 0, oL = oH + al(p->band_elems), oR = oL + al(nsig_L), oE = oR + al(nsig_R),
               oG = oE + al(nE), o1 = oG + al(nE * p->band_elems), oI = o1 + al(nE * b0 * bN),
               need = oI + al(nE);
  if (!p->host_io || p->host_io_bytes < need) {
    drop_graph(p);   // a captured host-copy schedule refers to the old buffers
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
  const bool overlap = p->n_domains == 1 && host_pinned(G_band) && host_pinned(G_1N);
  if (overlap) {
    e = ensure_copy_streams(p);
    if (e != cudaSuccess) return cuda_status(e);
    CallKey key{};
    key.kind = CALL_SOLVE_HOST;
    key.stride = sigma_E_stride;
    const void* ptrs[] = {G_band, G_1N, dL, dR};
    std::memcpy(key.p, ptrs, sizeof(ptrs));
    negf_status s = run_captured(p, key, [&]() -> cudaError_t {
      return solve_body(p, dH, dL, dR, sigma_E_stride, dE, dG, d1, dI, G_band, G_1N);
    });
    if (s != NEGF_OK) return s;
  } else {
    negf_status s = negf_solve(p, dH, dL, dR, sigma_E_stride, dE, dG, d1, dI);
    if (s != NEGF_OK) return s;
    if (G_band) e = cudaMemcpyAsync(G_band, dG, (size_t)(nE * p->band_elems) * z, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && G_1N) e = cudaMemcpyAsync(G_1N, d1, (size_t)(nE * b0 * bN) * z, cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(info, dI, (size_t)nE * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_status(e);
  return negf_sync(p);
}

// Keldysh equation for the selected blocks (see Sweep::lesser_up / down).
negf_status negf_lesser(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L, const negf_c128* sigma_R,
                        int64_t sigma_E_stride, const negf_c128* E, const negf_c128* sigma_less_L,
                        const negf_c128* sigma_less_R, int64_t sless_stride, const negf_c128* less_diag,
                        negf_c128* G_band, negf_c128* G_less, int32_t* info) {
  if (!p || !H || !E || !info || !G_band || !G_less || bad_sigma_stride(p, sigma_E_stride) ||
      bad_sigma_stride(p, sless_stride))
    return NEGF_ERR_ARG;
  if (!(p->outputs & NEGF_OUT_LESSER)) return NEGF_ERR_ARG;
  if (p->w > 1)
    return p->fz ? fused_lesser(p, (const double2*)H, (const double2*)sigma_L, (const double2*)sigma_R, sigma_E_stride,
                                (const double2*)E, (const double2*)sigma_less_L, (const double2*)sigma_less_R,
                                sless_stride, (const double2*)less_diag, (double2*)G_band, (double2*)G_less, info)
                 : NEGF_ERR_UNSUPPORTED;
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
  if (!p || !H || !E || !G_band || !res || bad_sigma_stride(p, sigma_E_stride)) return NEGF_ERR_ARG;
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
  double per_k[NEGF_AUTOTUNE_CANDIDATES];
  negf_status st = NEGF_OK;
  for (int k = 0; k < NEGF_AUTOTUNE_CANDIDATES; ++k) {
    per_k[k] = -1.0;
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
    per_k[k] = per;
    if (per < best_ms) best_ms = per;
  }
  // the fewest groups within 1 % of the fastest: fewer, larger launches for
  // the same time, and on negf_solve_host fewer copy streams (measured on
  // 64 x 64 x 512 energies: 4 and 6 groups both 136.8 ms on the device,
  // 137.2 and 144.4 ms with the band copied back to host memory)
  for (int k = 0; k < NEGF_AUTOTUNE_CANDIDATES && st == NEGF_OK; ++k)
    if (per_k[k] >= 0.0 && per_k[k] <= 1.01 * best_ms) { best = cand[k]; best_ms = per_k[k]; break; }
  p->groups = st == NEGF_OK ? best : g0;
  // mixed plans: the tensor-core products' N tile at that group count, from
  // the widest the tensor memory holds (one CTA may take all 512 columns of
  // an SM) or half of it (two CTAs hold tensor memory at once; A is sliced
  // once per tile): which is faster depends on the block sizes and widths
  if (st == NEGF_OK && p->precision == NEGF_MIXED) {
    const int c0 = p->tc_cols;
    int best_c = c0;
    double best_c_ms = best_ms;
    for (int cols : {512, 256}) {
      if (cols == c0) continue;
      p->tc_cols = cols;
      drop_graph(p);
      st = negf_solve(p, H, sigma_L, sigma_R, sigma_E_stride, E, G_band, G_1N, info);
      if (st != NEGF_OK) break;
      if (cudaEventRecord(a, p->stream) != cudaSuccess) { st = NEGF_ERR_CUDA; break; }
      for (int r = 0; r < reps && st == NEGF_OK; ++r)
        st = negf_solve(p, H, sigma_L, sigma_R, sigma_E_stride, E, G_band, G_1N, info);
      if (st != NEGF_OK) break;
      float t = 0.0f;
      if (cudaEventRecord(b, p->stream) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
          cudaEventElapsedTime(&t, a, b) != cudaSuccess) { st = NEGF_ERR_CUDA; break; }
      const double per = (double)t / reps;
      if (per < best_c_ms) { best_c_ms = per; best_c = cols; }
    }
    p->tc_cols = st == NEGF_OK ? best_c : c0;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  drop_graph(p);
  if (best_groups) *best_groups = p->groups;
  return st;
}

int32_t negf_plan_tile_cols(const negf_plan_t* p) { return p ? p->tc_cols : -1; }

negf_status negf_plan_set_tile_cols(negf_plan_t* p, int32_t cols) {
  if (!p || (cols != 512 && cols != 256)) return NEGF_ERR_ARG;
  if (cols != p->tc_cols) {
    p->tc_cols = cols;
    drop_graph(p);
  }
  return NEGF_OK;
}

int32_t negf_plan_groups(const negf_plan_t* p) { return p ? p->groups : -1; }

int32_t negf_plan_product_bits(const negf_plan_t* p) { return p ? p->bits : -1; }

// Precision tuner: a reference solve at 56 bits, then the candidate widths
// from the narrowest; the first whose band and G_1N stay within tol of the
// reference at every energy (relative Frobenius norm per energy and output)
// is kept for the plan's later calls.
negf_status negf_tune_precision(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                                const negf_c128* sigma_R, int64_t sigma_E_stride, const negf_c128* E,
                                negf_c128* G_band, negf_c128* G_1N, int32_t* info, negf_c128* G_band_ref,
                                negf_c128* G_1N_ref, double tol, int32_t* bits_out, double* dev_out) {
  if (!p || !H || !E || !info || !(tol > 0.0) || (!G_band && !G_1N)) return NEGF_ERR_ARG;
  if ((G_band && !G_band_ref) || (G_1N && !G_1N_ref)) return NEGF_ERR_ARG;
  if (p->precision != NEGF_MIXED) return NEGF_ERR_UNSUPPORTED;
  const int cand[NEGF_TUNE_BITS_CANDIDATES] = {32, 35, 42, 48};   // 4, 5, 6 and 7 slices
  const int nE = p->nE;
  const int64_t s1 = (int64_t)p->b[0] * p->b[p->N - 1];
  double* d = nullptr;   // per-energy squared norms: band diff, band ref, G_1N diff, G_1N ref
  cudaError_t ce = cudaMalloc((void**)&d, sizeof(double) * 4 * (size_t)nE);
  if (ce != cudaSuccess) { g_last_cuda = ce; cudaGetLastError(); return NEGF_ERR_NOMEM; }
  std::vector<double> h(4 * (size_t)nE);
  const int bits0 = p->bits;
  auto solve_at = [&](int bits, negf_c128* gb, negf_c128* g1) -> negf_status {
    if (p->bits != bits) { p->bits = bits; drop_graph(p); }
    negf_status st = negf_solve(p, H, sigma_L, sigma_R, sigma_E_stride, E, gb, g1, info);
    return st != NEGF_OK ? st : negf_sync(p);
  };
  negf_status st = solve_at(56, G_band_ref, G_1N_ref);
  int best = 56;
  double best_dev = 0.0;
  for (int k = 0; k < NEGF_TUNE_BITS_CANDIDATES && st == NEGF_OK; ++k) {
    st = solve_at(cand[k], G_band, G_1N);
    if (st != NEGF_OK) break;
    ce = cudaSuccess;
    if (G_band) {
      ce = negf::frob2_diff((const double2*)G_band, p->band_elems, (const double2*)G_band_ref, p->band_elems,
                            p->band_elems, d, nE, p->stream);
      if (ce == cudaSuccess)
        ce = negf::frob2((const double2*)G_band_ref, p->band_elems, p->band_elems, d + nE, nE, 0, p->stream);
    }
    if (ce == cudaSuccess && G_1N) {
      ce = negf::frob2_diff((const double2*)G_1N, s1, (const double2*)G_1N_ref, s1, s1, d + 2 * nE, nE, p->stream);
      if (ce == cudaSuccess) ce = negf::frob2((const double2*)G_1N_ref, s1, s1, d + 3 * nE, nE, 0, p->stream);
    }
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h.data(), d, sizeof(double) * 4 * nE, cudaMemcpyDeviceToHost, p->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(p->stream);
    if (ce != cudaSuccess) { st = cuda_status(ce); break; }
    double dev = 0.0;
    for (int e = 0; e < nE; ++e) {
      if (G_band) dev = std::max(dev, std::sqrt(h[e] / std::max(h[nE + e], 1e-300)));
      if (G_1N) dev = std::max(dev, std::sqrt(h[2 * nE + e] / std::max(h[3 * nE + e], 1e-300)));
    }
    if (dev < tol) { best = cand[k]; best_dev = dev; break; }
  }
  cudaFree(d);
  if (st != NEGF_OK) best = bits0;
  if (p->bits != best) { p->bits = best; drop_graph(p); }
  if (bits_out) *bits_out = best;
  if (dev_out) *dev_out = best_dev;
  return st;
}

negf_status negf_plan_set_groups(negf_plan_t* p, int32_t groups) {
  if (!p || groups < 1 || groups > (int)p->side.size() + 1) return NEGF_ERR_ARG;
  if (groups != p->groups) {
    if (p->n_domains > 1) return NEGF_ERR_UNSUPPORTED;   // per-group domain streams are fixed
    p->groups = groups;
    drop_graph(p);
  }
  return NEGF_OK;
}

negf_status negf_plan_set_wait_limit(negf_plan_t* p, int64_t polls) {
  if (!p) return NEGF_ERR_ARG;
  const long long v = polls < 0 ? -1 : (long long)polls;
  if (v != p->wait_limit) {
    p->wait_limit = v;
    drop_graph(p);   // the limit is a kernel argument of the captured schedule
  }
  return NEGF_OK;
}

negf_status negf_profile_enable(negf_plan_t* p, int32_t on) {
  if (!p) return NEGF_ERR_ARG;
  p->profiling = on != 0;
  return NEGF_OK;
}

int32_t negf_profile_read_issued(negf_plan_t* p, double* ms, double* flops, double* issued_flops,
                                 int64_t* launches) {
  if (!p) return -1;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return -1;
  for (auto& r : p->recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      p->prof_ms[r.kind] += t;
      p->prof_flops[r.kind] += r.flops;
      p->prof_issued[r.kind] += r.issued;
      p->prof_launches[r.kind] += 1;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  p->recs.clear();
  for (int k = 0; k < NEGF_PROF_KINDS; ++k) {
    if (ms) ms[k] = p->prof_ms[k];
    if (flops) flops[k] = p->prof_flops[k];
    if (issued_flops) issued_flops[k] = p->prof_issued[k];
    if (launches) launches[k] = p->prof_launches[k];
    p->prof_ms[k] = 0; p->prof_flops[k] = 0; p->prof_issued[k] = 0; p->prof_launches[k] = 0;
  }
  return NEGF_PROF_KINDS;
}

int32_t negf_profile_read(negf_plan_t* p, double* ms, double* flops, int64_t* launches) {
  return negf_profile_read_issued(p, ms, flops, nullptr, launches);
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
  if (!H || !E || !info || (!G_band && !G_1N)) return NEGF_ERR_ARG;
  if (bad_sigma_stride_sizes(d->block_sizes[0], d->block_sizes[d->n_blocks - 1], sigma_E_stride))
    return NEGF_ERR_ARG;
  if (d->n_domains != 1 || d->precision != NEGF_FP64 || (d->outputs & ~(NEGF_OUT_BAND | NEGF_OUT_G1N)))
    return NEGF_ERR_UNSUPPORTED;
  // every requested output needs its buffer
  if (((d->outputs & NEGF_OUT_BAND) && !G_band) || ((d->outputs & NEGF_OUT_G1N) && !G_1N)) return NEGF_ERR_ARG;
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
