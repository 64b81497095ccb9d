/*
 * ladder.h -- C ABI of the GB300 particle-particle ladder library (libladder.so).
 *
 * The library evaluates the closed-shell particle-particle ladder term of
 * Cholesky-based CCSD (Sec. "Acceleration of CC calculations", Eq. ppl-term
 * with Eq. cholesky inserted, i.e. Eq. vfunction-chol):
 *
 *     R[i,j,a,b] += sum_{c,d} (ac|bd) t2[i,j,c,d],
 *     (ac|bd)     = sum_P L[P,a,c] L[P,b,d],
 *
 * rebuilding (ac|bd) on the fly from the Cholesky vectors in blocks of
 * (a, b) pairs sized to the device memory (Sec. "Memory Management",
 * "An Asymmetric and Dynamic Splitting Protocol", Table 1).  Only pairs with
 * a <= b are formed; R_ji^ba = R_ij^ab supplies the rest.
 *
 * Index roles follow the paper's 'xac,xbd,icjd' contraction with the output
 * stored (i, j, a, b) and the amplitudes stored (i, j, c, d).
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Arrays are C-contiguous (row-major) IEEE float64 in device memory of the
 *   plan's device:  L[nchol][nv][nv], t2[no][no][nv][nv], R[no][no][nv][nv].
 *   Device pointers must be 256-byte aligned, otherwise LADDER_ERR_ARG.
 * - Precondition ASSUMED, not checked: t2[i,j,a,b] == t2[j,i,b,a].  The
 *   a <= b packing relies on it (with a non-symmetric t2 the result differs
 *   from the definition).  The emulated path (LADDER_EMU_BF16) also assumes
 *   L[P,a,c] == L[P,c,a], as Cholesky vectors of (ac|bd) with real orbitals
 *   are: it multiplies only the rows (a <= c) of L^T and takes the entries
 *   where a row meets itself from squared norms.  The FP64 path needs no
 *   symmetry of L.
 * - Ownership: the caller owns L, t2, R and the workspace.  A plan owns only
 *   host metadata and a small device table written at plan time.
 * - ladder_apply / ladder_apply_batched perform no allocation and no host
 *   synchronisation; all work is enqueued on the given stream.
 * - Synchronous errors (bad arguments, CUDA launch failures) are returned.
 *   Errors detected by kernels (a bounded wait that ran out, a failed
 *   consistency check) are recorded in the plan's device status word and
 *   reported by ladder_last_status().
 * - Not provided: no CPU fallback and no backend selection.
 */
#ifndef LADDER_H
#define LADDER_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ladder_plan_s* ladder_plan_t;

/* Status codes. */
enum {
    LADDER_OK = 0,
    LADDER_ERR_ARG = 1,          /* invalid argument, size, alignment or null pointer   */
    LADDER_ERR_BUDGET = 2,       /* no blocking fits the workspace budget                */
    LADDER_ERR_CUDA = 3,         /* a CUDA runtime / driver call failed                  */
    LADDER_ERR_UNSUPPORTED = 4,  /* valid request this build does not implement          */
    LADDER_ERR_TIMEOUT = 5,      /* a kernel's bounded wait ran out (device status)      */
    LADDER_ERR_NUMERIC = 6,      /* a kernel consistency check failed (device status)    */
    LADDER_ERR_BOUNDS = 7        /* an index check of a LADDER_CHECK build failed         */
};

/* Arithmetic of the two contractions. */
enum {
    LADDER_FP64 = 0,      /* native FP64 (DMMA tensor instructions)                        */
    LADDER_EMU_BF16 = 1,  /* FP64 emulated by BF16 digit slices on tcgen05, FP32 accumulate */
    LADDER_EMU_INT8 = 2   /* INT8 slices: rejected with LADDER_ERR_UNSUPPORTED             */
};

/*
 * ladder_plan -- choose the blocking and the kernels for one problem shape.
 *
 * Defines: the a/b blocking of the (a <= b) pair space (Sec. "An Asymmetric
 * and Dynamic Splitting Protocol", Table 1, the C-split loop nest).  Blocks of
 * n_a virtual indices a and n_b indices b (n_a != n_b allowed) are chosen by
 * a cost model subject to the workspace budget.
 *
 *   out        receives the plan handle (set to NULL on failure).
 *   no, nv     occupied / virtual orbital counts (>= 1).
 *   nchol      number of Cholesky vectors (>= 1).
 *   precision  LADDER_FP64 or LADDER_EMU_BF16.
 *   nslices    digit slices per operand for the emulated path, 0 = default (6);
 *              ignored for LADDER_FP64.  Valid range 5..8.
 *   ws_budget_bytes  workspace budget; 0 = 0.9 * 0.98 * free device memory
 *              (the safety factors of the paper's C-split rule).
 *   device     CUDA device ordinal.
 *
 * Returns LADDER_OK, LADDER_ERR_ARG, LADDER_ERR_BUDGET (no blocking fits),
 * LADDER_ERR_UNSUPPORTED (LADDER_EMU_INT8) or
 * LADDER_ERR_CUDA.  Allocates a small device table (freed by
 * ladder_plan_destroy).
 */
int ladder_plan(ladder_plan_t* out, int no, int nv, int nchol, int precision, int nslices,
                size_t ws_budget_bytes, int device);

/* Force the a/b block sizes of an existing plan (tests, tuning).  Rebuilds the
 * device tables.  Returns LADDER_ERR_BUDGET if the workspace would exceed the
 * plan's budget, LADDER_ERR_ARG for sizes outside 1..nv. */
int ladder_plan_set_blocks(ladder_plan_t plan, int n_a, int n_b);

/*
 * ladder_plan_set_form -- arithmetic form of the emulated ladder GEMM of a plan.
 *   0 (default): K = (c,d) over all c, d and rows = all (i,j), as in Eq. vfunction-chol.
 *   1: symmetric/antisymmetric split.  With t_ij^cd = t_ji^dc the sum is taken over
 *      c <= d only, as X_ij^ab = sum_{c<=d} V'_ab,cd T'_ij,cd (i <= j) and
 *      Y_ij^ab = sum_{c<d} V''_ab,cd T''_ij,cd (i < j), with V' = V_cd + V_dc (V_cc on the
 *      diagonal), V'' = V_cd - V_dc, T' = (T_ij,cd + T_ji,cd)/2 (T_ij,cc), T'' = (T_ij,cd -
 *      T_ji,cd)/2, and R_ij^ab += X + Y, R_ji^ab += X - Y: half the multiply-adds of the
 *      ladder GEMM, for one extra pass per block pair that reads V (kept as int64 in this
 *      form) and writes the V' and V'' digit planes (re-sliced with the pair's exponent bound
 *      plus one, one rounding of half a unit).  K' and K'' are packed in 4-byte words of two
 *      (c,d) slots, a few zero slots per row included.  This split is not in the paper.
 * The blocking is kept if its workspace still fits the plan's budget, else chosen again.
 * Call before querying the workspace.  Returns LADDER_OK, LADDER_ERR_ARG (batched plan or a
 * form other than 0, 1), LADDER_ERR_UNSUPPORTED (form 1 on the FP64 path), LADDER_ERR_BUDGET
 * or LADDER_ERR_CUDA.
 */
int ladder_plan_set_form(ladder_plan_t plan, int form);
/* The form a plan uses: ladder_plan picks 1 on the emulated path when a cost model of the whole
 * call (ERI, tile-padded ladder rows, the extra pass over V) gives it a 5 % lead (the ladder a
 * large share of the call: large no^2 with respect to the 128/256-row MMA tiles and to nchol)
 * and the workspace fits, else 0.  The instances of a batched plan choose the same way.  -1 for
 * NULL. */
int ladder_plan_get_form(ladder_plan_t plan);
/* The form the cost model above picks for an emulated plan of this shape (nslices 0 = the
 * default), before the workspace check: 0 or 1; -1 for invalid arguments.  Host only. */
int ladder_form_model(int no, int nv, int nchol, int nslices);

/*
 * ladder_plan_set_path -- evaluation order of a plan (Sec. "Acceleration of CC calculations":
 * the ladder term can be evaluated by rebuilding (ac|bd) from the Cholesky vectors, 2 x v^4 work
 * per vector, or by contracting the amplitudes with one Cholesky factor at a time, x o^2 v^3
 * work per factor; which is cheaper depends on x against o^2 and on v against o^2).
 *   LADDER_PATH_ERI (0): (ac|bd) rebuilt per (A,B) block pair of a <= b pairs, then the ladder
 *     GEMM: 2 nchol nv^2 p + 2 no^2 nv^2 p flops (p = nv(nv+1)/2).
 *   LADDER_PATH_FACTORISED (1): R_ij = sum_P L_P T_ij L_P^T over the amplitude pairs i <= j
 *     (R_ji = R_ij^T from t_ji^cd = t_ij^dc), as two FP64 DMMA GEMMs per batch of Cholesky
 *     vectors through a workspace W[o(o+1)/2][nv][batch][nv]: 4 nchol o(o+1)/2 nv^3 flops.
 *     Native FP64 plans only (LADDER_ERR_UNSUPPORTED for the emulated path).
 *   LADDER_PATH_FUSED (2): the rebuild order with the two C-split steps of a batch kept on the
 *     chip (Sec. "An Asymmetric and Dynamic Splitting Protocol", Table 1, steps 0 and 1): one
 *     kernel per block pair builds (ac|bd) for a tile of 4 x 4 pairs (a, b) one 16 x 16 chunk of
 *     (c, d) at a time into shared memory and contracts each chunk with t2 at once into
 *     accumulators for all no^2 amplitude rows held in registers; V is never written.  Same
 *     flops as path 0 (plus the pairs a > b of the tiles that straddle the diagonal), no
 *     workspace beyond the minimum (ladder_workspace_bytes returns 256), one block pair of all
 *     pairs unless the plan is a shard.  Native FP64 plans with no^2 <= 1024 only
 *     (LADDER_ERR_UNSUPPORTED otherwise).
 * ladder_plan picks, for an FP64 plan, the factorised path when it needs 1.25x fewer flops and its
 * workspace fits, else the fused path when no^2 <= 1024 (same flops as path 0 without the V round
 * trip), else path 0; and the fused path whenever no workspace of the others fits.  Emulated
 * plans use path 0.  Forcing a blocking (ladder_plan_set_blocks) returns a
 * plan to path 0; sharding (ladder_plan_shard) returns a factorised plan to path 0 and splits the
 * block pairs of a fused plan.
 * Returns LADDER_OK, LADDER_ERR_ARG, LADDER_ERR_UNSUPPORTED, LADDER_ERR_BUDGET (path 1: the batch
 * of one Cholesky vector does not fit; path 0: no blocking fits) or LADDER_ERR_CUDA; on an error
 * the plan keeps its path.  ladder_plan_get_path: the plan's path, -1 for NULL.
 * ladder_path_model: host only, the path ladder_plan would pick for this shape and precision
 * before the workspace check (0, 1 or 2; -1 for invalid arguments).
 */
enum { LADDER_PATH_ERI = 0, LADDER_PATH_FACTORISED = 1, LADDER_PATH_FUSED = 2 };
int ladder_plan_set_path(ladder_plan_t plan, int path);
int ladder_plan_get_path(ladder_plan_t plan);
int ladder_path_model(int no, int nv, int nchol, int precision);

/*
 * Data-parallel sharding over several GPUs (the multi-GPU direction named in
 * Sec. "Conclusions and outlook"; the sharding itself is this library's).
 * The (A,B) block pairs of one contraction are independent: each writes the
 * entries R_ij^ab of its own pairs a <= b and their mirrors R_ji^ba, which no
 * other block pair touches, so ranks that each run a share of the block pairs
 * on their own GPU produce disjoint parts of R with no exchange, and E_L (linear
 * in R) is the sum of the ranks' ladder_energy values (one scalar all-reduce).
 *
 * ladder_shard_blocks -- host only: owner[k] in [0, world) for each of n_blocks
 *   block pairs with pair counts npairs[k]: largest first (ties by position),
 *   each to the least-loaded rank (ties: lower rank).  LADDER_ERR_ARG for
 *   world < 1, n_blocks < 0 or NULL arrays.
 *
 * ladder_plan_shard -- restrict `plan` to the block pairs that rank `rank` of
 *   `world` owns.  If the plan has fewer than 2*world block pairs (and the
 *   shape allows more) the planner first re-selects the blocking under the same
 *   budget with at least that many.  All ranks must build their plans with the
 *   same shape, precision, slices and an explicit equal ws_budget_bytes, so that
 *   they see the same blocking.  The workspace size may shrink (query it again).
 *   A rank may own no block pair; its ladder_apply then leaves R unchanged.
 *   Call once per plan (a second call, or ladder_plan_set_blocks afterwards,
 *   returns LADDER_ERR_ARG); world == 1 is a no-op.  Not for batched plans.
 */
int ladder_shard_blocks(int n_blocks, const long long* npairs, int world, int* owner);
int ladder_plan_shard(ladder_plan_t plan, int rank, int world);

/*
 * ladder_plan_dry -- run the planner on the host only (no CUDA call), for
 * inspection and tests.  Same meaning of no, nv, nchol, precision, nslices as
 * ladder_plan; ws_budget_bytes must be > 0 and num_sms >= 1 (the SM count the
 * cost model assumes).  force_n_a / force_n_b > 0 impose block sizes instead
 * of the model's choice.  Outputs (any may be NULL): chosen n_a, n_b, the
 * workspace bytes, the number of (A,B) block pairs, and up to max_blocks rows
 * of blocks[5*k..5*k+4] = {a0, a1, b0, b1, npairs} in execution order.
 * Returns LADDER_OK, LADDER_ERR_ARG, LADDER_ERR_BUDGET or LADDER_ERR_UNSUPPORTED.
 *
 * ladder_plan_shard_dry -- the same host-only planner followed by the selection that
 * ladder_plan_shard makes for rank `rank` of `world` (block pairs re-selected when fewer than
 * 2*world, then the longest-first partition): outputs as above, for the rank's own block pairs
 * (the workspace bytes are its shard's).  LADDER_ERR_ARG also for rank outside [0, world).
 */
int ladder_plan_shard_dry(int no, int nv, int nchol, int precision, int nslices, size_t ws_budget_bytes, int num_sms,
                          int rank, int world, int* n_a, int* n_b, size_t* ws_bytes, int max_blocks,
                          int* n_block_pairs, int* blocks);
int ladder_plan_dry(int no, int nv, int nchol, int precision, int nslices, size_t ws_budget_bytes, int num_sms,
                    int force_n_a, int force_n_b, int* n_a, int* n_b, size_t* ws_bytes, int max_blocks,
                    int* n_block_pairs, int* blocks);

/*
 * ladder_watchdog_selftest -- check, on the current device, the bounded wait that every
 * tcgen05 kernel of the library uses for its mbarriers (the watchdog that turns a lost
 * producer into LADDER_ERR_TIMEOUT instead of a hang).  Launches one CTA on `stream` that
 * waits on an mbarrier nothing arrives on, with that same wait (limit: limit_s seconds of the
 * GPU's global timer, 0 = the plans' default of 2 s; at most 60 s, else LADDER_ERR_ARG), then
 * synchronises the stream.  Returns LADDER_ERR_TIMEOUT when the wait
 * gave up and reported it through its status word -- the expected outcome -- and stores the
 * time it waited in *waited_ms (may be NULL); LADDER_OK means the wait ended without the
 * timeout being reported (a broken watchdog); LADDER_ERR_CUDA on a CUDA error.  Allocates and
 * frees 16 bytes of device memory.  The paper's failure handling is a CUDA availability probe
 * with a CPU fallback (Sec. "A Generic Interface for a Dynamic Switching Between CuPy,
 * PyTorch, and CPU-only Libraries"); this library has no fallback and no counterpart there.
 */
int ladder_watchdog_selftest(double limit_s, double* waited_ms, cudaStream_t stream);

/* Workspace bytes ladder_apply needs (device memory, 256-byte aligned start). */
size_t ladder_workspace_bytes(ladder_plan_t plan);

/* Describe a plan: block sizes, number of (A,B) block pairs, largest pair
 * count of a block, slices.  Any output pointer may be NULL. */
int ladder_plan_describe(ladder_plan_t plan, int* n_a, int* n_b, int* n_block_pairs,
                         int* max_pairs_per_block, int* nslices, int* precision);

/*
 * ladder_apply -- R += ladder(L, t2)   (Eq. vfunction-chol).
 *
 *   L   device, [nchol][nv][nv] float64.
 *   t2  device, [no][no][nv][nv] float64, t2[i,j,a,b] == t2[j,i,b,a].
 *   R   device, [no][no][nv][nv] float64, accumulated in place (+=).
 *   ws  device workspace of ladder_workspace_bytes(plan) bytes (contents
 *       need not be initialised; they are overwritten).
 *   stream  CUDA stream; all work is enqueued on it, nothing synchronises.
 *
 * Returns LADDER_OK or LADDER_ERR_ARG / LADDER_ERR_CUDA.  L, t2 and R must not
 * overlap each other or the workspace.
 */
int ladder_apply(ladder_plan_t plan, const double* L, const double* t2, double* R, void* ws,
                 cudaStream_t stream);

/*
 * ladder_apply_host -- R_host = ladder(L_host, t2_host)   (Eq. vfunction-chol), for operands in
 * host memory: the inputs are copied to the device, R is formed there from zero (not
 * accumulated into R_host) and copied back.  The paper's engine stages host arrays to the GPU
 * and back around every batch (Sec. "An Asymmetric and Dynamic Splitting Protocol"); here the
 * copies of one call overlap the contraction of the previous one.
 *
 *   L_host   host, [nchol][nv][nv] float64;  t2_host host, [no][no][nv][nv] float64 (symmetric
 *            as for ladder_apply);  R_host host, [no][no][nv][nv] float64, written.
 *   stage    device buffer of ladder_host_staging_bytes(plan) bytes (256-byte aligned): two
 *            sets of device copies of L, t2 and R.  Successive calls on a plan alternate between
 *            the sets.  A call enqueues its host-to-device copies on a copy stream the plan owns,
 *            behind an event of the call two back (the last one to use the same set), so they
 *            run while the previous call computes; the contraction waits for them on `stream`,
 *            then the device-to-host copy of R follows on `stream`.
 *   ws       the workspace of ladder_apply;  stream  the caller's stream.
 *
 * R_host holds the result once `stream` has reached the end of the call (e.g. after
 * cudaStreamSynchronize(stream)); L_host and t2_host must stay unchanged until then.  Pinned
 * host memory (cudaHostAlloc / cudaHostRegister) lets the copies run asynchronously; pageable
 * memory works but the copies then block the host.  Successive calls on one plan must use the
 * same stream, and the same stage buffer.  The first call creates the plan's copy stream and
 * four events (freed with the plan), so it cannot be captured into a graph; no call is
 * capturable, since the copy stream is not part of the caller's capture.  For a shard plan
 * R_host receives the shard's entries (zero elsewhere).  Returns LADDER_OK, LADDER_ERR_ARG
 * (NULL pointer, misaligned stage or ws, batched plan), LADDER_ERR_CUDA, or what ladder_apply
 * returns.  ladder_host_staging_bytes: 0 for NULL or a batched plan.
 */
size_t ladder_host_staging_bytes(ladder_plan_t plan);
int ladder_apply_host(ladder_plan_t plan, const double* L_host, const double* t2_host, double* R_host,
                      void* stage, void* ws, cudaStream_t stream);

/*
 * ladder_energy -- E_L = sum_{ijab} (2 t2[i,j,a,b] - t2[i,j,b,a]) R[i,j,a,b].
 *
 * The closed-shell energy expression the ladder residual enters (the CC energy
 * evaluation of Sec. "Molecular benchmark calculations").  FP64 throughout,
 * fixed-order tree reduction (deterministic).
 *
 *   E_dev   device double* receiving E_L, or NULL.
 *   E_host  host double* receiving E_L, or NULL; when non-NULL the call
 *           synchronises the stream to read the value back.
 * At least one of E_dev / E_host must be non-NULL.
 */
int ladder_energy(ladder_plan_t plan, const double* t2, const double* R, double* E_dev,
                  double* E_host, cudaStream_t stream);

/*
 * ladder_plan_batched -- one plan for n independent ladder instances of
 * uneven shape (no[k], nv[k], nchol[k]), run by ladder_apply_batched (the
 * batching of independent contractions that the paper's engine does one after
 * another, Sec. "A Generic Batching Recipe").  Each instance gets its own
 * sub-plan against the whole budget (one block pair whenever its packed ERI
 * fits).  The plan's workspace (ladder_workspace_bytes) holds as many
 * instances at once as the budget allows.  Two kinds of schedule:
 *   grouped (emulated path, the default): the instances are packed, largest
 *     workspace first, into groups that fit the workspace, of at most 32
 *     instances and 32 ladder items (one per instance in the plain form, X
 *     and Y in the symmetric/antisymmetric one; an instance whose Cholesky
 *     vectors are sliced in batches is a group of its own); each group runs as
 *     ONE persistent ERI launch over the tiles of all its instances, the
 *     combine pass of each split-form instance, then ONE persistent ladder
 *     launch per ladder shape (single CTAs for up to 128 rows, CTA pairs
 *     above) over all their items' units, with the small per-instance
 *     preparation and finalisation kernels around them;
 *   worker streams (the FP64 path's default): each instance runs as its own
 *     ladder_apply on one of k plan-owned streams (longest first).
 * ladder_batched_schedule selects one explicitly, ladder_tune_batched by
 * measurement.  Same precision / nslices / budget / device meaning as
 * ladder_plan.
 */
int ladder_plan_batched(ladder_plan_t* out, int n, const int* no, const int* nv, const int* nchol,
                        int precision, int nslices, size_t ws_budget_bytes, int device);

/*
 * ladder_batched_schedule -- set the schedule of a batched plan.  schedule > 0:
 * that many worker streams (at most the number that fit the workspace, and 8);
 * schedule < 0: grouped, with at most ws_bytes / |schedule| of workspace per
 * group (emulated path only).  Returns LADDER_OK, LADDER_ERR_ARG (not a batched
 * plan, schedule 0, grouped on the FP64 path), LADDER_ERR_BUDGET (an instance
 * does not fit the group size) or LADDER_ERR_CUDA.  *groups_or_streams (may be
 * NULL) receives the resulting number of groups (negated) or streams.
 */
int ladder_batched_schedule(ladder_plan_t plan, int schedule, int* groups_or_streams);

/*
 * ladder_apply_batched -- R[k] += ladder(L[k], t2[k]) for every instance k.
 * L, t2, R are HOST arrays of n device pointers.  Grouped schedule: everything
 * is enqueued on `stream`.  Worker-stream schedule: the instances run on the
 * plan's streams, forked from and joined back into `stream` with events.
 * No allocation and no host synchronisation: the whole call can be captured
 * into one CUDA graph from `stream`.
 */
int ladder_apply_batched(ladder_plan_t plan, const double* const* L, const double* const* t2,
                         double* const* R, void* ws, cudaStream_t stream);

/*
 * ladder_tune_batched -- measured tuner of a batched plan: times
 * ladder_apply_batched under worker-stream schedules with 1, 2, 4, ... streams
 * and (emulated path) grouped schedules with the whole workspace, a half and a
 * quarter of it per group (the batch splits), each with the one-SM ladder tile
 * widths 96 and 64 (emulated path; ladder_plan_set_ladder_tile), on the given
 * buffers, and keeps the fastest.  R[k]
 * is accumulated into by every trial (pass scratch R).  Synchronises the
 * stream.  *best_schedule (may be NULL) receives the chosen schedule: the
 * number of streams (> 0) or minus the number of groups (< 0).
 */
int ladder_tune_batched(ladder_plan_t plan, const double* const* L, const double* const* t2,
                        double* const* R, void* ws, cudaStream_t stream, int* best_schedule);

/*
 * ladder_plan_set_pbatch -- slice the Cholesky vectors a batch of pb at a time (emulated path;
 * the P-split of a blocked Cholesky contraction).  The L^T digit planes of all nchol vectors take
 * 2 nslices bytes per element of L for the whole call; with batches only pb vectors' planes are
 * resident, sliced again for every (A,B) block pair, and the ERI of each batch adds its exact int64
 * sums into V (every batch uses the exponents of all the vectors, so the sums share one fixed-point
 * unit); the last batch rounds V onto the pair's grid.  This needs the symmetric/antisymmetric
 * form's int64 V, so a plan with batches uses form 1.  ladder_plan picks batches of 8192, 4096,
 * 2048 or 1024 vectors when a cost model (larger blocks against re-slicing L per block pair)
 * prefers them or when nothing else fits the budget.  pb = 0 (or >= nchol) slices all vectors at
 * once; otherwise pb must be a multiple of 64.  The exact levels of the ERI do not depend on the
 * batches (see ladder_plan_set_eri_chunk for the shared tail level).  Returns LADDER_OK,
 * LADDER_ERR_ARG (batched or sharded plan, bad pb), LADDER_ERR_UNSUPPORTED (pb > 0 on the FP64
 * path), LADDER_ERR_BUDGET or LADDER_ERR_CUDA.  ladder_plan_get_pbatch: the batch, 0 for none,
 * -1 for NULL.  ladder_plan_set_form(plan, 0) is refused (LADDER_ERR_ARG) while batches are set.
 */
int ladder_plan_set_pbatch(ladder_plan_t plan, int pb);
int ladder_plan_get_pbatch(ladder_plan_t plan);

/*
 * ladder_plan_set_eri_chunk -- longest exact K chunk of the emulated ERI, in blocks of 1024
 * Cholesky vectors (1..4, default 4).  Each chunk ends with a drain of the tensor-memory
 * accumulators into int64 registers that the next chunk's MMAs wait for.  With |digit| <= 64 a
 * chunk of 1024 keeps every exact level sum an FP32 integer for any data; longer chunks are taken,
 * per call and on the device, only when a bound from the operands' own digits proves the same:
 * by Cauchy-Schwarz each level-l sum over a chunk is at most sum_{s+t=l-2} M_s M_t, M_s the
 * largest 2-norm of slice s's digits over any L^T row within one chunk-aligned window, and the
 * longest window (up to the limit) whose bounds stay within (l-1) 2^22 for l = 2..5 is used.  The
 * exact levels do not depend on the chunk; the shared accumulator of the levels >= 6 (weight
 * <= 2^-28 of the leading level) is rounded once per chunk, which can move the int64 sum of an
 * ERI element by a few units of 2^-49 of its scale before it is rounded to the V grid (2^-42), so
 * results agree to that level (bit for bit in the tested cases).  blocks = 1 keeps 1024.  Applies
 * to a batched plan's instances too.  Returns LADDER_OK or LADDER_ERR_ARG.
 *
 * ladder_plan_eri_chunk -- the chunk length (Cholesky vectors) the last ladder_apply of an emulated
 * plan with workspace `ws` chose; synchronises `stream` to read it.  -1 for a NULL, batched, FP64
 * or factorised plan or a failed read.
 */
int ladder_plan_set_eri_chunk(ladder_plan_t plan, int blocks);
int ladder_plan_eri_chunk(ladder_plan_t plan, const void* ws, cudaStream_t stream);

/*
 * ladder_plan_set_ladder_tile -- column tile of the emulated ladder GEMM when it runs on one SM
 * (no^2 <= 128 amplitude rows; the CTA-pair form keeps 96): bn pairs per tile, a multiple of 16
 * in [16, 96] (96 is the widest the five TMEM accumulators leave room for: 5 x bn <= 512
 * columns).  Narrower tiles make more, smaller units for instances with few pairs.
 * The result does not depend on it (exact integer accumulation).  Applies to a batched plan's
 * instances too; ladder_tune_batched measures 96 and 64 with every schedule and keeps the best.
 * Returns LADDER_OK or LADDER_ERR_ARG.  ladder_plan_get_ladder_tile: the width, -1 for NULL.
 */
int ladder_plan_set_ladder_tile(ladder_plan_t plan, int bn);
int ladder_plan_get_ladder_tile(ladder_plan_t plan);

/*
 * Per-kernel timing for benchmarks.  ladder_plan_set_timing(plan, 1) creates a
 * pool of CUDA events; while enabled, ladder_apply records an event pair on
 * its stream around the launches of each kernel class, tagged with the class
 * (LADDER_KERNEL_*).  ladder_plan_timing waits for the recorded events and
 * returns, for one class, the summed elapsed milliseconds and the number of kernels launched
 * since the last reset; reset != 0 clears all records afterwards.  Timing is
 * off by default and costs nothing then.
 */
enum {
    LADDER_KERNEL_PREP = 0,     /* operand slicing / exponent kernels (emulated path) */
    LADDER_KERNEL_ERI = 1,      /* Cholesky -> ERI GEMM                               */
    LADDER_KERNEL_LADDER = 2,   /* ladder GEMM                                        */
    LADDER_KERNEL_FINISH = 3,   /* accumulator finalisation / unpack                  */
    LADDER_KERNEL_COMBINE = 4,  /* V' and V'' from V (symmetric/antisymmetric form)   */
    LADDER_KERNEL_FACT_W = 5,   /* factorised path: W = L_P T_ij                      */
    LADDER_KERNEL_FACT_R = 6,   /* factorised path: R_ij += W L_P^T                   */
    LADDER_KERNEL_FUSED = 7,    /* fused path: ERI chunks contracted on chip          */
    LADDER_KERNEL_CLASSES = 8
};
int ladder_plan_set_timing(ladder_plan_t plan, int enable);
int ladder_plan_timing(ladder_plan_t plan, int kernel_class, float* total_ms, int* launches, int reset);

/*
 * ladder_plan_set_wait_limit -- time limit of the bounded waits in the plan's tensor-core
 * kernels (and, for a batched plan, its instances').  Every mbarrier wait of those kernels polls
 * the GPU's global nanosecond timer and gives up after this long: the kernel then records
 * LADDER_ERR_TIMEOUT in the plan's status word, waits (bounded) for its own copies and MMAs,
 * frees its tensor memory and returns, so a lost producer never hangs the GPU.  A stage can
 * legitimately wait longer than the default 2 s on a time-sliced GPU or under a profiler's
 * replay; raise the limit for such runs.  seconds = 0 restores the default; otherwise it must
 * lie in [0.001, 3600].  Takes effect for calls enqueued afterwards.  Returns LADDER_OK or
 * LADDER_ERR_ARG.  ladder_plan_get_wait_limit returns the limit in seconds (-1 for NULL).
 * This failure handling is the library's own: the paper's is a CUDA availability probe with a
 * CPU fallback (Sec. "A Generic Interface for a Dynamic Switching Between CuPy, PyTorch, and
 * CPU-only Libraries").
 */
int ladder_plan_set_wait_limit(ladder_plan_t plan, double seconds);
double ladder_plan_get_wait_limit(ladder_plan_t plan);

/* Read (and clear) the plan's device status word: LADDER_OK, LADDER_ERR_BOUNDS
 * (only in a library built with LADDER_CHECK, whose kernels test the index of
 * every store into the workspace and into R, record a failure here and skip the
 * store), LADDER_ERR_TIMEOUT or LADDER_ERR_NUMERIC.  Synchronises the stream.
 * After LADDER_ERR_TIMEOUT or LADDER_ERR_NUMERIC the R of the calls enqueued since the last
 * read is undefined (partly accumulated, or built from clamped digits): restore R and repeat
 * the call.  The workspace needs no repair; the context stays usable. */
int ladder_last_status(ladder_plan_t plan, cudaStream_t stream);

/*
 * ladder_energy_noalloc -- the E_L of ladder_energy (same definition), for
 * callers that cannot allocate device memory.  The paper has no counterpart
 * to this entry point.  Its fixed reduction tree (contiguous runs of 64 tiles)
 * differs from ladder_energy's, so the two may differ by rounding; for a given
 * (no, nv) and data every call returns the same bits.
 *
 * Who needs it: code that runs while a stream is being captured into a CUDA
 * graph (allocation cannot be captured), frameworks that own all device
 * memory through their own pool and forbid other allocators, and loops that
 * must not take the allocator's locks.  It needs no plan and no workspace
 * and calls no cudaMalloc, cudaFree or allocating library routine.
 *
 *   no, nv  orbital counts (>= 1); t2, R device [no][no][nv][nv] float64 on
 *           the current device; E_dev device double receiving E_L.
 *   stream  CUDA stream; the call enqueues two kernels and does not wait.
 *
 * Scratch: a 128 KiB file-scope device array (LADDER_NOALLOC_MAX_PARTIALS
 * doubles) that every device loading the library holds until the process
 * exits.  One partial sum per 64 tiles of 32 x 32 (a, b) elements, so the
 * call rejects, with LADDER_ERR_ARG and before launching anything, shapes
 * with ceil(no^2 ceil(nv/32)^2 / 64) > LADDER_NOALLOC_MAX_PARTIALS.
 * The first call on a device looks up the array's device address with that
 * device current (again after cudaDeviceReset, or under another driver
 * context of the device); make that first call before any stream capture.  All calls
 * share the one array: calls whose kernels may overlap on the GPU (other
 * streams, other threads) race and return wrong values -- order them.
 * Every partial is rewritten by each call, so nothing is cleared in between.
 * Returns LADDER_OK, LADDER_ERR_ARG or LADDER_ERR_CUDA.
 */
#define LADDER_NOALLOC_MAX_PARTIALS 16384
int ladder_energy_noalloc(int no, int nv, const double* t2, const double* R, double* E_dev,
                          cudaStream_t stream);

/* Release a plan (NULL is ignored).  Frees the plan's device table. */
void ladder_plan_destroy(ladder_plan_t plan);

/* Static, human-readable description of a status code. */
const char* ladder_strerror(int status);

/* Algorithmic FP64 flop count of one ladder_apply with a <= b packing:
 * 2 nchol nv^2 p + 2 no^2 nv^2 p, p = nv (nv + 1) / 2. */
double ladder_flops(int no, int nv, int nchol);

#ifdef __cplusplus
}
#endif

#endif /* LADDER_H */
