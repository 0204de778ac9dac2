/*
 * negf.h -- C-ABI of the GB300 selected-inversion library (libnegf.so).
 *
 * The library computes, for a grid of complex energies E, selected blocks of
 * the retarded Green's function
 *
 *     G^R(E) = M(E)^{-1},   M(E) = E I - H - Sigma^R            (Sec. 2, eq. for M)
 *
 * where H is block n-diagonal over N principal layers (n = 3, 5, ...; the
 * half-bandwidth is w = (n-1)/2, Sec. 2.3, Prop. 3) and the lead
 * self-energy Sigma^R acts on layer 1 (Sigma_L) and layer N (Sigma_R) only.
 * The selected blocks are bndiag(G^R) (Sec. 2, "the Dyson problem"), computed
 * by the recursive Green's function method (Alg. 1; Sec. 2.3 for n > 3) or by
 * single-level domain-decomposition RGF (Alg. 2), plus the corner block
 * G_{1N} (Eq. 4x4_exact_RGF, first row), the transmission
 * T(E) = Tr[Gamma_L G_1N Gamma_R G_1N^H] with Gamma = i(Sigma - Sigma^H), and
 * the gradient of T with respect to the band blocks of H and to Sigma_L/R.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Complex numbers are interleaved (re, im) doubles: negf_c128, the layout
 *   of cuDoubleComplex and of torch.complex128.
 * - Every block is dense and row-major: block (i, j) has b_i rows and b_j
 *   columns, element (r, c) at offset r * b_j + c.
 * - "Band-packed" storage of a block n-diagonal matrix: the existing blocks
 *   (i, i + d) are stored back to back for d = -w .. w (outer) and
 *   i = 0 .. N-1 (inner), skipping blocks with i + d outside [0, N).
 *   negf_band_offset() gives the element offset of block (i, i + d) and
 *   negf_band_elems() the total element count of one band-packed matrix.
 *   Layers are 0-based in this interface.
 * - All array arguments of negf_solve / negf_transmission / negf_grad are
 *   DEVICE pointers on the device that was current at negf_plan().  The
 *   caller owns them; the library never frees them.  Calls are asynchronous
 *   on the plan's stream: outputs are ready after negf_sync() or after any
 *   later work on that stream.
 * - Errors: argument errors are returned before anything is launched.
 *   Numerical failures found on the device (an exactly zero or non-finite
 *   pivot in a per-block inversion) are written to info[e] (0 = success,
 *   k > 0 = 1-based layer whose Schur complement failed first, for energy e)
 *   and folded into the status that negf_sync() returns
 *   (NEGF_ERR_SINGULAR / NEGF_ERR_NONFINITE).  No entry point aborts,
 *   traps or throws.
 * - A plan is not thread-safe; use one plan per host thread.
 */
#ifndef NEGF_H
#define NEGF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } negf_c128;

typedef enum {
  NEGF_OK = 0,
  NEGF_ERR_ARG = 1,          /* invalid argument or descriptor                */
  NEGF_ERR_SINGULAR = 2,     /* a zero pivot in a per-block inversion          */
  NEGF_ERR_NONFINITE = 3,    /* a NaN/Inf pivot (e.g. NaN in H)                */
  NEGF_ERR_NOMEM = 4,        /* workspace allocation failed                    */
  NEGF_ERR_CUDA = 5,         /* a CUDA runtime call failed                     */
  NEGF_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up             */
  NEGF_ERR_UNSUPPORTED = 7   /* valid request this library does not implement  */
} negf_status;

/* Arithmetic of the sweep.
 * NEGF_FP64:  every product and every per-block inverse in double precision.
 * NEGF_MIXED: block products on the tensor cores from exact BF16 slices
 *             (each operand cut into integer slices below a power-of-two
 *             scale per row / column, every slice product and FP32 sum exact;
 *             negf_desc.product_bits significant bits,
 *             NEGF_DEFAULT_PRODUCT_BITS by default), per-block inverses in
 *             FP64; inputs and outputs stay complex128.  DDRGF plans
 *             (n_domains > 1) keep the interface system in FP64. */
typedef enum { NEGF_FP64 = 0, NEGF_MIXED = 1 } negf_precision;

/* Output selection bits (negf_desc.outputs). */
enum {
  NEGF_OUT_BAND = 1,          /* bndiag(G) per energy                          */
  NEGF_OUT_G1N = 2,           /* G_{1N} per energy                             */
  NEGF_OUT_TRANSMISSION = 4,  /* T(E)                                          */
  NEGF_OUT_GRAD = 8,          /* allow negf_grad (keeps the first-row chain)   */
  NEGF_OUT_LESSER = 16        /* allow negf_lesser (keeps W_i, g^<_i per layer) */
};

typedef struct {
  int32_t n_blocks;                   /* N >= 1 (N > w)                        */
  const int32_t* block_sizes;         /* host array of N sizes b_i, 1 <= b_i <= NEGF_MAX_BLOCK */
  int32_t band_n;                     /* n = 3 or 5 (w = (n-1)/2)              */
  int32_t n_energies;                 /* >= 1                                  */
  int32_t n_domains;                  /* 1 = plain RGF, >1 = DDRGF pairs,
                                         0 = chosen with the interface levels
                                         by negf_ddrgf_model from a measured
                                         r_inv (plain RGF for plans with
                                         NEGF_OUT_GRAD)
                                         (Alg. 2): sub-domain sweeps in the
                                         plan's precision, interface Schur
                                         system and its RGF in FP64            */
  const int32_t* domain_first_block;  /* host, n_domains entries or NULL: first
                                         layer of each (D2, D1) pair; pair j is
                                         D2_j then a separator D1_j of w layers;
                                         entry 0 must be 0, every pair must have
                                         at least 3w layers.  NULL balances the
                                         pairs by sum of b_i^3 (Sec. 3).        */
  int32_t precision;                  /* negf_precision                        */
  int32_t refine_steps;               /* 0 or 1 (NEGF_MIXED only)              */
  int32_t outputs;                    /* NEGF_OUT_* bit mask                   */
  int32_t checkpoint_every;           /* adjoint plans (NEGF_OUT_GRAD): 0 keeps
                                         the whole forward factorisation of an
                                         energy chunk; k > 0 keeps rings of k + 1
                                         layers and one checkpoint (S_i, P_i) per
                                         segment of k layers, and negf_grad
                                         recomputes each segment (one extra
                                         upward sweep; memory ~ (N/k + 3k) blocks
                                         per energy instead of ~6N).  Such a plan
                                         serves negf_transmission and G_1N-only
                                         negf_solve; a band request returns
                                         NEGF_ERR_UNSUPPORTED.  Ignored without
                                         NEGF_OUT_GRAD.  < 0: NEGF_ERR_ARG.     */
  int32_t product_bits;               /* NEGF_MIXED: significant bits of the
                                         tensor-core block products, 16..56
                                         (0 = NEGF_DEFAULT_PRODUCT_BITS, which
                                         meets 1e-5 on chains with localised
                                         states at eta = 1e-6;
                                         negf_tune_precision narrows it where
                                         the caller's inputs allow); more bits
                                         trade speed for accuracy.  Products
                                         too long for exact slices at that
                                         width (K x slices beyond the FP32
                                         sums) run as FP64 DMMA products.
                                         DDRGF plans form the closed
                                         sub-domains' corner blocks with
                                         56-bit products whatever the width. */
  int32_t n_levels;                   /* DDRGF plans: levels of the interface
                                         recursion below the first (0 = the
                                         separators' chain by sequential
                                         sweeps, Alg. 2 step 3 "via RGF")    */
  const int32_t* level_domains;       /* host, n_levels entries or NULL:
                                         level k + 2 cuts the previous level's
                                         chain of separators into
                                         level_domains[k] pairs (a group of
                                         separators, then one separator; at
                                         least 2 per pair), balanced by count
                                         (Alg. 2 step 3 "recursive DDRGF",
                                         s_1 = 1 below the first level)       */
} negf_desc;

#define NEGF_MAX_BLOCK 160
#define NEGF_DEFAULT_PRODUCT_BITS 48
#define NEGF_TUNE_BITS_CANDIDATES 4   /* widths negf_tune_precision tries: 32 35 42 48 */
#define NEGF_MAX_GROUPS 8   /* energy groups (concurrent streams) per plan */
#define NEGF_AUTOTUNE_CANDIDATES 6   /* group counts negf_autotune times: 1 2 3 4 6 8 */

typedef struct negf_plan_s negf_plan_t;   /* opaque plan handle */

/* Validate the descriptor, fix the schedule and allocate the workspace.
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream).
 * Returns NEGF_ERR_ARG for an invalid descriptor, NEGF_ERR_NOMEM if the
 * workspace cannot be allocated, NEGF_ERR_UNSUPPORTED for a combination this
 * build does not implement.  On success *out owns the workspace. */
negf_status negf_plan(negf_plan_t** out, const negf_desc* d, void* cuda_stream);

/* Bytes of device workspace the plan holds.  negf_plan sizes it to
 * max(24 GiB, 45 % of the device memory free at plan time) and runs the
 * energies in chunks that fit; the environment variable NEGF_WORKSPACE_GB
 * (a positive number, read by negf_plan) caps it instead (at least one
 * energy per chunk). */
size_t negf_workspace_bytes(const negf_plan_t* p);

/* The plan's number of DDRGF (D2, D1) pairs (1 = plain RGF); -1 for NULL. */
int32_t negf_plan_n_domains(const negf_plan_t* p);

/* The plan's interface levels below the first (their count, or -1 for NULL);
 * up to cap pair counts into level_domains (nullable). */
int32_t negf_plan_levels(const negf_plan_t* p, int32_t* level_domains, int32_t cap);

/* The paper's DDRGF cost model (Sec. 3, Eq. cost_model_DDRGF with Eq.
 * cost_model_RGF) evaluated for a GPU; pure host arithmetic.  Costs are in
 * units of one batched block product: r_RGF(l) = l (4 + r_LU + 3 r_GETRS) -
 * (4 + 2 r_GETRS) with r_LU = r_inv (the measured ratio of a batched block
 * inversion to a batched block product, negf_measure_r_inv) and r_GETRS = 1
 * (products with explicit inverses are products); the paper's
 * n_tasks / n_threads becomes the wave factor
 * max(1, n_tasks n_E / slots, n_tasks / 16) (slots: inversion CTAs resident
 * on sm_count SMs for the largest block; concurrent tasks are graph branches
 * of latency-bound launches, of which about 16 progress at once on GB300,
 * measured).
 * Level 1 pairs have s2 in {2, 3, 4, 6, ..., 128} w layers and s1 = w
 * separator layers and at most 128 pairs (one graph branch per pair);
 * deeper levels s2 in {1, 2, 3, 4}, s1 = 1 (the paper's
 * auto-tuner table), up to max_levels levels below the first, each level's
 * Schur complement holding l_S = n_tasks s1 nodes, n_tasks = floor(l /
 * (s1 + s2)) (the paper rounds up; here every pair holds a whole group and
 * its separator).  Returns the pair count
 * of the cheapest choice (1 = plain RGF); level_domains (nullable, up to
 * max_levels entries) / n_levels receive the deeper levels' pair counts;
 * cost_rgf / cost_ddrgf (nullable): the two model costs.  1 for invalid
 * arguments. */
int32_t negf_ddrgf_model(int32_t n_blocks, const int32_t* block_sizes, int32_t band_n, int32_t n_energies,
                         int32_t sm_count, double r_inv, int32_t max_levels, int32_t* level_domains,
                         int32_t* n_levels, double* cost_rgf, double* cost_ddrgf);

/* Measures r_inv for b x b blocks on the current device with the library's
 * own kernels: the CUDA-event time of a batched FP64 inversion of `batch`
 * blocks over that of a batched block product of the same blocks in the
 * given precision (NEGF_MIXED: tensor-core products at the default width),
 * 10 repetitions each after 3 warm-ups.  The result is also cached for
 * negf_plan's n_domains = 0 choice.  Allocates and frees its operands;
 * synchronous on cuda_stream (NULL = legacy default stream). */
negf_status negf_measure_r_inv(int32_t b, int32_t batch, int32_t precision, double* r_inv, void* cuda_stream);

/* RGF / DDRGF choice made for n_domains = 0 (pure host arithmetic, no device
 * call).  Cost model: a layer step over x independent block problems costs
 * max(lat, thr x / slots) latency-bound RGF layer steps, slots = inversion
 * CTAs resident on sm_count SMs for the largest block.  Plain RGF: N steps
 * over n_E problems (lat = thr = 1).  DDRGF with d (D2, D1) pairs: N/d steps
 * over d n_E concurrent sub-domain problems (lat 4.5, thr 15: the extended
 * sweep's extra launches and work, fitted to GB300 runs), then the interface
 * RGF, d steps over n_E problems at w^3 the work.  Returns 1 or the power of
 * two d >= 2 (pairs of at least 4w layers) of least cost; 1 for invalid
 * arguments.  The paper recommends independent RGF runs when they fill the
 * machine and DDRGF otherwise, with an "orchestrator" to choose (Sec. 4,
 * DDRGF results, closing paragraphs). */
int32_t negf_auto_domains(int32_t n_blocks, const int32_t* block_sizes, int32_t band_n, int32_t n_energies,
                          int32_t sm_count);

/* Element offset of block (i, i + d) in band-packed storage, or -1 if that
 * block does not exist (|d| > w or i + d outside [0, N)). */
int64_t negf_band_offset(const negf_plan_t* p, int32_t d, int32_t i);

/* Elements of one band-packed matrix (per energy). */
int64_t negf_band_elems(const negf_plan_t* p);

/* bndiag(G^R(E)) and/or G_{1N} for every energy (Alg. 1, Sec. 2.3, Alg. 2).
 *   H:       band-packed H (energy independent), negf_band_elems() elements.
 *   sigma_L: b_1 x b_1 per energy, energy e at sigma_L + e * sigma_E_stride
 *            (stride 0 broadcasts one matrix to all energies); same for sigma_R
 *            (b_N x b_N).  sigma_E_stride is in elements: 0, or at least
 *            max(b_1^2, b_N^2) (smaller strides are NEGF_ERR_ARG).
 *   E:       n_energies complex energies (E_r + i eta).
 *   G_band:  n_energies x negf_band_elems() elements (energy-major); may be
 *            NULL if NEGF_OUT_BAND is not requested.
 *   G_1N:    n_energies x (b_1 * b_N); may be NULL.
 *   info:    n_energies int32 (see the error conventions above); required. */
negf_status negf_solve(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                       const negf_c128* sigma_R, int64_t sigma_E_stride,
                       const negf_c128* E, negf_c128* G_band, negf_c128* G_1N,
                       int32_t* info);

/* T(E) = Tr[Gamma_L G_1N Gamma_R G_1N^H] for every energy into T[n_energies]
 * (doubles).  Same inputs as negf_solve. */
negf_status negf_transmission(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                              const negf_c128* sigma_R, int64_t sigma_E_stride,
                              const negf_c128* E, double* T, int32_t* info);

/* Gradient of L = sum_e dL_dT[e] * T(E_e) (vector-Jacobian product) with
 * respect to the band blocks of H and to sigma_L / sigma_R, in the
 * convention dL/dRe z + i dL/dIm z (the one torch.autograd uses for a real
 * loss of complex inputs).  Blocks of H are treated as independent inputs
 * (the Hermitian tie H_{i+1,i} = H_{i,i+1}^H is not imposed).
 *   dL_dT:    n_energies doubles.
 *   T:        optional (may be NULL): receives T(E) as in negf_transmission.
 *   dH:       band-packed, negf_band_elems() elements, summed over energies.
 *   dSigma_L: b_1 x b_1 per energy with stride sigma_E_stride (0 = summed
 *             over energies into one matrix); dSigma_R likewise.  Either may
 *             be NULL.
 * Requires a plan with NEGF_OUT_GRAD.  DDRGF plans (n_domains > 1) run it on
 * a plain RGF sub-plan of the same chain (the gradient of T does not depend
 * on the method that solved for it).  Block n-diagonal plans (band_n >= 5)
 * run it on their fused block tridiagonal chain (a
 * sub-plan on w-layer super-blocks, within NEGF_MAX_BLOCK; checkpoint_every
 * applies there): the fused H is the band laid out on super-blocks, so each
 * band block's gradient is its sub-block of the super-block's gradient, and
 * info[e] is the first layer of a failing w-layer group. */
negf_status negf_grad(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                      const negf_c128* sigma_R, int64_t sigma_E_stride,
                      const negf_c128* E, const double* dL_dT, double* T,
                      negf_c128* dH, negf_c128* dSigma_L, negf_c128* dSigma_R,
                      int32_t* info);

/* negf_grad with separate output strides for the self-energy gradients:
 * dSigma_L at dSigma_L + e * dSigma_L_stride (0 = summed over energies into
 * one matrix), dSigma_R likewise, independently of sigma_E_stride (a lead
 * given once for all energies can have per-energy gradients and the other
 * way round).  Each output stride is 0 or at least max(b_1^2, b_N^2)
 * (otherwise NEGF_ERR_ARG).  negf_grad is this call with both output strides
 * equal to sigma_E_stride. */
negf_status negf_grad_strided(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                              const negf_c128* sigma_R, int64_t sigma_E_stride, const negf_c128* E,
                              const double* dL_dT, double* T, negf_c128* dH, negf_c128* dSigma_L,
                              int64_t dSigma_L_stride, negf_c128* dSigma_R, int64_t dSigma_R_stride,
                              int32_t* info);

/* negf_solve with the caller's buffers in HOST memory (same arguments and
 * layouts as negf_solve, every pointer a host pointer): the inputs are
 * copied to device buffers the plan owns (allocated at the first call, kept
 * for later ones: band_elems + the self-energies + n_energies x (band_elems
 * + b_1 b_N) elements), the solve runs as negf_solve, and G_band / G_1N /
 * info are copied back, all on the plan's stream.  Synchronous: returns when
 * the outputs are in host memory, with negf_sync's status.  Page-locked host
 * memory (cudaHostAlloc, torch pin_memory) lets the copies run at the link's
 * rate; pageable memory works, more slowly.  With page-locked G_band / G_1N
 * on a plain RGF plan (n_domains == 1) the copies back overlap the solve:
 * each energy group copies its band in pieces of layers as its downward
 * pass completes them, on a copy stream of its own, and its G_1N after that.
 * NEGF_ERR_NOMEM if the device buffers cannot be allocated;
 * NEGF_ERR_UNSUPPORTED for a band on a checkpointed adjoint plan. */
negf_status negf_solve_host(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                            const negf_c128* sigma_R, int64_t sigma_E_stride, const negf_c128* E,
                            negf_c128* G_band, negf_c128* G_1N, int32_t* info);

/* Selected blocks of the Keldysh equation G^< = G^R Sigma^< G^A (Sec. 1; the
 * paper leaves its recursive solution to future work, Sec. 5), plain RGF
 * plans (n_domains = 1) with NEGF_OUT_LESSER.  Block n-diagonal plans
 * (band_n >= 5) run it on their fused block tridiagonal chain (Sec. 2.3:
 * super-layers of w layers, which must stay within NEGF_MAX_BLOCK): the band
 * of H and the leads are laid out on the super-blocks by block copies, the
 * recursion below runs there (the plan keeps a sub-plan for that, with the
 * plan's precision and product width at plan time, and device buffers for
 * at most ~8 GiB of fused outputs per sub-call), and both bands are cut
 * back; there info[e] is the first layer of the failing w-layer group.  Runs
 * the retarded sweep (written to G_band) and a recursion over the
 * factorisation M = U D L of its upward pass:
 *   upward   Q_i = Sigma^<_i + H_{i,i+1} g^<_{i+1} H_{i,i+1}^H,
 *            W_i = Q_i t_i^H, g^<_i = t_i W_i   (right-connected lesser),
 *   downward G^<_11 = g^<_1, A_i = G^R_{i-1,i} W_i,
 *            G^<_{i,i-1} = -X_{i,i-1} G^<_{i-1,i-1} - A_i^H,
 *            G^<_{i-1,i} = -(G^<_{i,i-1})^H,
 *            G^<_ii = g^<_i - X_{i,i-1} A_i - G^<_{i,i-1} X_{i,i-1}^H,
 * X_{i,i-1} = t_i M_{i,i-1}.  The layer-local lesser self-energy is
 *   Sigma^<_1 = sigma_less_L + s_e I,  Sigma^<_N = sigma_less_R + s_e I,
 *   Sigma^<_i = s_e I otherwise,
 * with sigma_less_L / _R (b_1^2 / b_N^2 per energy at sless_stride elements,
 * 0 broadcasts; nullable) and less_diag = n_energies complex scalars s_e
 * (nullable; e.g. 2 i eta f for the broadening's own reservoir).
 * G_band: the retarded band (required, as negf_solve writes it); G_less: the
 * lesser band, same band packing (required).  All products in the plan's
 * precision.  Errors as negf_solve; NEGF_ERR_ARG for a plan without
 * NEGF_OUT_LESSER. */
negf_status negf_lesser(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                        const negf_c128* sigma_R, int64_t sigma_E_stride, const negf_c128* E,
                        const negf_c128* sigma_less_L, const negf_c128* sigma_less_R,
                        int64_t sless_stride, const negf_c128* less_diag, negf_c128* G_band,
                        negf_c128* G_less, int32_t* info);

/* A-posteriori accuracy of a band from the band alone (no oracle, no
 * off-band block): the diagonal blocks of M G - I,
 *   R_i = sum_{|c - i| <= w} M_{i,c} G_{c,i} - I,   M = E I - H - Sigma,
 *   res[e] = sqrt( sum_i ||R_i||_F^2 / sum_i b_i ),
 * with FP64 products.  G_band: n_energies band-packed matrices as written by
 * negf_solve; res: n_energies doubles (device).  Asynchronous on the plan's
 * stream like negf_solve; uses the plan's workspace, so it must not overlap
 * another call on the same plan.  0 for the exact band; a band with relative
 * error r typically gives res of order r * ||M|| ||G||. */
negf_status negf_band_residual(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                               const negf_c128* sigma_R, int64_t sigma_E_stride, const negf_c128* E,
                               const negf_c128* G_band, double* res);

/* Energy-group autotuner.  A plan splits the energies of a chunk into
 * groups that run concurrently on forked streams (graph branches), so that
 * one group's tensor-core products overlap another's inversions.  This call
 * replays the plan's negf_solve schedule on the caller's buffers (same
 * arguments as negf_solve) with 1, 2, 3, 4, 6 and 8 groups (at most
 * NEGF_MAX_GROUPS, at most one group per energy of a chunk), `reps` timed
 * repetitions each after one warm-up, and keeps for the plan's later calls
 * the fewest groups whose time is within 1 % of the fastest.  ms (nullable): NEGF_AUTOTUNE_CANDIDATES doubles, the
 * time per solve for each candidate in that order, or -1 where skipped.  best_groups (nullable): the kept count.
 * Mixed plans then time the tensor-core products' N tile at that count: the
 * widest tile whose level accumulators fit an SM's 512 tensor-memory columns,
 * or the widest within 256 (two CTAs hold tensor memory at once, the A
 * operand is sliced once per tile), and keep the faster (negf_plan_tile_cols).
 * Synchronises the plan's stream.  NEGF_ERR_UNSUPPORTED for DDRGF and
 * checkpointed plans (fixed stream sets). */
negf_status negf_autotune(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                          const negf_c128* sigma_R, int64_t sigma_E_stride, const negf_c128* E,
                          negf_c128* G_band, negf_c128* G_1N, int32_t* info, int32_t reps,
                          int32_t* best_groups, double* ms);

/* Precision tuner (mixed plans): solves the caller's inputs once with
 * 56-bit products into G_band_ref / G_1N_ref (caller-owned device buffers of
 * the outputs' sizes), then with 32, 35, 42 and 48 bits (4 to 7 slices) into G_band / G_1N,
 * and keeps for the plan's later calls the narrowest width whose band and
 * G_1N lie within tol of the 56-bit reference at every energy (relative
 * Frobenius norm per energy and output kind); 56 if none does.  The choice
 * holds for inputs like the tuned ones: re-tune when H, Sigma or the
 * energies change in kind.  bits_out / dev_out (nullable): the kept width
 * and its largest deviation.  Allocates 4 n_energies doubles for the
 * duration of the call; synchronises the plan's stream.
 * NEGF_ERR_UNSUPPORTED for an FP64 plan. */
negf_status negf_tune_precision(negf_plan_t* p, const negf_c128* H, const negf_c128* sigma_L,
                                const negf_c128* sigma_R, int64_t sigma_E_stride, const negf_c128* E,
                                negf_c128* G_band, negf_c128* G_1N, int32_t* info, negf_c128* G_band_ref,
                                negf_c128* G_1N_ref, double tol, int32_t* bits_out, double* dev_out);

/* The plan's product width in bits (0 for FP64 plans); -1 for NULL. */
int32_t negf_plan_product_bits(const negf_plan_t* p);

/* The tensor-memory columns one tensor-core product CTA of the plan may take
 * (512 or 256, set by negf_autotune); -1 for NULL. */
int32_t negf_plan_tile_cols(const negf_plan_t* p);

/* Set it for later calls (512 or 256, else NEGF_ERR_ARG). */
negf_status negf_plan_set_tile_cols(negf_plan_t* p, int32_t cols);

/* The plan's current number of energy groups; -1 for NULL. */
int32_t negf_plan_groups(const negf_plan_t* p);

/* Set the number of energy groups of later calls (1 .. the count the plan's
 * streams allow: NEGF_MAX_GROUPS, at most one per energy of a chunk; DDRGF
 * plans keep theirs).  The next call captures a new graph.  NEGF_ERR_ARG for
 * a count out of range, NEGF_ERR_UNSUPPORTED for changing a DDRGF plan. */
negf_status negf_plan_set_groups(negf_plan_t* p, int32_t groups);

/* Bound of the tensor-core product kernel's wait for its MMAs (the one
 * device-side wait of the library: polls of mbarrier.try_wait per K chunk,
 * after which the kernel stops, drains the MMAs already issued with the
 * default bound, frees its tensor memory, records NEGF_ERR_TIMEOUT in the
 * plan's error word and leaves that product unwritten).  For tests of the
 * timeout path (polls = 0 makes every wait run out at once) and for
 * callers that want a tighter watchdog.  polls < 0 restores the default
 * (2^26).  Later calls capture a new graph.  NEGF_ERR_ARG for NULL. */
negf_status negf_plan_set_wait_limit(negf_plan_t* p, int64_t polls);

/* Wait for the plan's stream, then return the first error the device
 * reported since the previous negf_sync (and clear it): a timeout first
 * (the products it left unwritten make later pivots meaningless), then a
 * non-finite pivot, then a singular one. */
negf_status negf_sync(negf_plan_t* p);

/* Release the workspace and the plan.  NULL is allowed. */
void negf_destroy(negf_plan_t* p);

/* Instrumentation: per-kernel timing of the calls made while enabled.
 * With profiling on, calls run without graph capture and every kernel launch
 * is bracketed by CUDA events on the plan's stream.  negf_profile_read waits
 * for the stream and returns, per kernel kind (index NEGF_PROF_*), the summed
 * device milliseconds, the algorithmic real flops (8 m n k per complex block
 * product, 8 b^3 per block inverse) and the launch count, then resets them.
 * Any of the three arrays may be NULL; each must hold NEGF_PROF_KINDS
 * entries.  Returns NEGF_PROF_KINDS, or -1 on error. */
enum { NEGF_PROF_INV = 0, NEGF_PROF_GEMM_F64 = 1, NEGF_PROF_GEMM_TC = 2, NEGF_PROF_MISC = 3,
       NEGF_PROF_KINDS = 4 };
negf_status negf_profile_enable(negf_plan_t* p, int32_t on);
int32_t negf_profile_read(negf_plan_t* p, double* ms, double* flops, int64_t* launches);
/* The same read (and reset), with the flops the hardware units execute per
 * kind as well (issued_flops, may be NULL): the inverse's 8 b^3; the FP64
 * product's three real products per complex one (3M form, 6 m n k); the
 * tensor-core product's BF16 slice products, L (L + 1) / 2 per 16-deep real
 * K step for L slices, over whole tiles of 128 real rows (padding included). */
int32_t negf_profile_read_issued(negf_plan_t* p, double* ms, double* flops, double* issued_flops,
                                 int64_t* launches);

/* negf_solve for callers that cannot allocate device memory.
 *
 * The paper has no counterpart: this entry point exists for embedding.  Some
 * callers cannot call cudaMalloc: code that runs while another component owns
 * all device memory through its own pool, code whose memory budget is fixed
 * before it runs, and loops that must not pay the device-wide
 * synchronisation an allocation can cause.  This call creates no plan and
 * allocates nothing on the device: its scratch (the per-block inverses, the
 * multipliers of the sweep and the running Schur complement) lives in one
 * file-scope device array of NEGF_NOALLOC_SCRATCH_BYTES bytes, which every
 * GPU that loads the library holds until the process exits.
 *
 * Arguments are those of negf_plan plus negf_solve, with the descriptor in
 * place of a plan: FP64 only, n_domains == 1, and outputs a subset of
 * NEGF_OUT_BAND | NEGF_OUT_G1N (anything else: NEGF_ERR_UNSUPPORTED; a
 * requested output with a NULL buffer: NEGF_ERR_ARG).  The caller passes
 * device inputs and outputs as for negf_solve, with the same rule on
 * sigma_E_stride (0, or at least max(b_1^2, b_N^2); else NEGF_ERR_ARG).  The
 * band is written when G_band is not NULL, G_1N when G_1N is not NULL.  If
 * the scratch this descriptor needs,
 *   256 + 16 * n_energies * (sum_i b_i^2 + 2 * sum_{|i-j|=1..w, i>j} b_i b_j
 *                            + (w+1)^2 * bmax^2 + (w+1) * b_1 * bmax)  bytes,
 * exceeds NEGF_NOALLOC_SCRATCH_BYTES, the call returns NEGF_ERR_ARG before
 * launching anything.  Work is enqueued on cuda_stream without a CUDA graph.
 * Numerical failures are reported only through info[] (there is no plan to
 * negf_sync): info[e] = k > 0 names the first layer (1-based) whose pivot
 * was zero OR non-finite; the two cases are not told apart here (a NaN or
 * Inf in H or Sigma shows as non-finite values in that energy's outputs).
 *
 * The first call on each device sets that device up (it looks up the device
 * address of the scratch array and sets kernel attributes); make that first
 * call before any stream capture.  Every call shares the one array and
 * leaves its contents behind: calls that overlap on the GPU (on different
 * streams, or from different host threads) race on it and must be
 * serialised by the caller. */
#define NEGF_NOALLOC_SCRATCH_BYTES (32u << 20)
negf_status negf_solve_noalloc(const negf_desc* d, const negf_c128* H, const negf_c128* sigma_L,
                               const negf_c128* sigma_R, int64_t sigma_E_stride, const negf_c128* E,
                               negf_c128* G_band, negf_c128* G_1N, int32_t* info, void* cuda_stream);

/* FP64 peak probe (instrumentation; no counterpart in the paper).  Runs one
 * kernel that keeps every SM's FP64 units busy with one instruction kind on
 * independent dependency chains, and returns the issued rate in TFLOP/s:
 *   NEGF_PEAK_DFMA: scalar FP64 fused multiply-add (2 flops each), the
 *                   arithmetic of the per-block inversion;
 *   NEGF_PEAK_DMMA: FP64 MMA m8n8k4 (512 flops per warp instruction), the
 *                   arithmetic of the FP64 block product;
 *   NEGF_PEAK_BOTH: half of the warps each (whether the two kinds share one
 *                   FP64 unit: the sum of both rates if they do not).
 * iters: loop trips per thread (8 instructions each; ~1e5 gives about
 * 0.1 s).  tflops: required; ms (nullable): the kernel's CUDA-event time.
 * Synchronous on cuda_stream (NULL = legacy default stream); allocates
 * nothing.  NEGF_ERR_ARG for an unknown kind or iters < 1. */
enum { NEGF_PEAK_DFMA = 0, NEGF_PEAK_DMMA = 1, NEGF_PEAK_BOTH = 2 };
negf_status negf_fp64_peak(int32_t kind, int32_t iters, double* tflops, double* ms, void* cuda_stream);

/* Text of the last CUDA runtime error this thread's calls met (for
 * NEGF_ERR_CUDA diagnostics); "no error" if none. */
const char* negf_last_cuda_error(void);

/* Static, human-readable name of a status code. */
const char* negf_status_string(negf_status s);

#ifdef __cplusplus
}
#endif
#endif /* NEGF_H */
