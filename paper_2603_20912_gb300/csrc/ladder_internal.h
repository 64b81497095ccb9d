// Internal definitions shared by the host-side runtime (planner, C ABI) and
// the kernel translation units.  Not part of the public interface.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ladder.h"

// Index checks of a LADDER_CHECK build: a store whose index fails `cond` records
// kStatusBounds in the status word and is skipped (no trap, no fault).  In a normal build the
// condition is not evaluated.
#ifdef LADDER_CHECK
#define LADDER_IN_BOUNDS(cond, status) \
    ((cond) ? true : (atomicOr((status), ::ladder::kStatusBounds), false))
#else
#define LADDER_IN_BOUNDS(cond, status) true
#endif

namespace ladder {

constexpr int kAlign = 256;                 // workspace sub-buffer alignment (bytes)
constexpr int kDefaultSlices = 6;           // digit slices per operand (emulated path)
constexpr int kDigitBits = 7;               // bits per signed digit, |digit| <= 64
constexpr int kExpGroupRows = 64;           // rows sharing one power-of-two exponent
constexpr int kEmuChunkK = 1024;            // K per exact chunk: level 5 has 4 pairs, 4 * 64^2 * K <= 2^24
constexpr int kEmuTile = 128;               // tcgen05 tile rows (M)
constexpr int kEmuTileN = 96;               // widest tile N: 5 TMEM accumulators x 96 <= 512 columns

// Default limit of the kernels' bounded mbarrier waits (ladder_plan_set_wait_limit changes it).
constexpr unsigned long long kDefaultWaitNs = 2000000000ull;   // 2 s

// Device status bits (ORed into the plan's status word by kernels).
constexpr unsigned kStatusTimeout = 1u;
constexpr unsigned kStatusNumeric = 2u;
constexpr unsigned kStatusBounds = 4u;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// One (A, B) block pair of the packed (a <= b) pair space: a in [a0, a1),
// b in [b0, b1).  Its valid pairs are numbered a-major, b-minor, skipping a > b.
struct BlockPair {
    int a0, a1, b0, b1;
    int npairs;        // number of (a, b) with a <= b in the block pair
    size_t pairs_off;  // offset (in int2) of this block pair's pair list in the device table
    size_t rows_off;   // offset (in int) of this block pair's row_start table (a1 - a0 + 1 ints)
    size_t tiles_off = 0;  // emulated path: offset (in int2) of the ERI entries (int4: rt, qt, 0, 0)
    int ntiles = 0;        // emulated path: number of ERI entries (one 2-CTA cluster each)
    size_t chunks_off = 0; // emulated path: offset (in int2) of the ERI row chunks (first L^T row, rows)
};

// Workspace layout of one plan (byte offsets from the workspace base).
struct WsLayout {
    size_t v_blk = 0;      // FP64: V block [max_pairs][nv*nv] f64; EMU: V slices [S][max_pairs][kpad] bf16
    size_t rp_int = 0;     // EMU: int64 fixed-point ladder accumulator [max_pairs][no*no]
    size_t lt_slices = 0;  // EMU: L^T slices [S][nv*nv][xpad] bf16
    size_t lt_exp = 0;     // EMU: exponent per group of L^T rows (int)
    size_t t_slices = 0;   // EMU: T slices [S][no*no][kpad] bf16
    size_t t_gmax = 0;     // EMU: max |T| per group of T rows (IEEE bits, u64)
    size_t t_exp = 0;      // EMU: exponent per group of T rows (int)
    size_t v_exp = 0;      // EMU: exponent bound per (a, b) pair [nv][nv] (int)
    size_t lnorm = 0;      // EMU: max_c ||L[:, a, c]||_2 per a (IEEE bits, u64)
    size_t lsq = 0;        // EMU: ||L[:, a, c]||_2^2 per (a, c) [nv][nv] (f64)
    size_t lt_norm2 = 0;   // EMU: squared digit norms of L^T [S][nv*vp][nblk] (u32), 1024-wide blocks of K
    size_t eri_cand = 0;   // EMU: largest windowed squared norms per (window length, plane) (u32)
    size_t eri_kbc = 0;    // EMU: K blocks per exact ERI chunk, chosen on the device (int)
    // EMU, symmetric/antisymmetric ladder form (instead of t_slices, t_gmax, t_exp, rp_int):
    size_t vp_blk = 0;     // V' planes [S][max_pairs][kp] bf16, K' = (c <= d) packed
    size_t vm_blk = 0;     // V'' planes [S][max_pairs][km] bf16, K'' = (c < d) packed
    size_t tp_slices = 0;  // T' planes [S][np][kp] bf16, rows (i <= j)
    size_t tm_slices = 0;  // T'' planes [S][nm][km] bf16, rows (i < j)
    size_t tp_gmax = 0, tm_gmax = 0;  // max |T'|, |T''| per group of rows (IEEE bits, u64)
    size_t tp_exp = 0, tm_exp = 0;    // exponent per group of rows (int)
    size_t rpx = 0, rpy = 0;          // int64 accumulators [max_pairs][np], [max_pairs][nm]
    // FP64 factorised path: W batch [o(o+1)/2][nv][fact_pb][nv] f64
    size_t w_blk = 0;
    size_t total = 0;
};

// Symmetric/antisymmetric ladder form: packed sizes of its K and row ranges.
// Padded (c, d) layout of the emulated path: vp = nv rounded up to 16, K index c * vp + d (zero
// for d >= nv).  With vp % 16 == 0 every pair of 8-column runs of a V row is one whole 32-byte
// sector, so V never leaves L2 half written.
inline int emu_vp(int nv) { return (nv + 15) / 16 * 16; }

// Packed (c,d) index of the symmetric (c <= d, plus) and antisymmetric (c < d) forms, in
// 4-byte words of two slots (d even, d + 1): row c holds the words that contain one of its
// elements, from d = c (plus) or c + 1 rounded down to even up to d = nv - 1, so element (c,d)
// sits in slot pm_base(c) + d with pm_base(c) even and every word belongs to one row; the slots
// without an element (d = c - 1 or c, d = nv) hold zero.  Rows of the antisymmetric form stop
// at c = nv - 2.  pm_words(c) is the first word of row c.
__host__ __device__ inline long long pm_words(int c, int nv, bool plus) {
    const long long h1 = (nv - 1) / 2 + 1;
    return plus ? (long long)c * h1 - (long long)(c / 2) * ((c - 1) / 2)
                : (long long)c * h1 - (long long)((c + 1) / 2) * (c / 2);
}
__host__ __device__ inline long long pm_base(int c, int nv, bool plus) {
    return 2 * (pm_words(c, nv, plus) - (plus ? c / 2 : (c + 1) / 2));
}

struct PmDims {
    long long kp, km;      // slots of the packed K' (c <= d) and K'' (c < d), pads included
    long long kp_pad, km_pad;  // rounded up to 8 (16-byte rows)
    int np, nm;            // rows: o(o+1)/2 (i <= j), o(o-1)/2 (i < j)
};
inline PmDims pm_dims(int no, int nv) {
    PmDims d;
    d.kp = 2 * pm_words(nv, nv, true);
    d.km = nv >= 2 ? 2 * pm_words(nv - 1, nv, false) : 0;
    d.kp_pad = (d.kp + 7) / 8 * 8;
    d.km_pad = (d.km + 7) / 8 * 8;
    d.np = no * (no + 1) / 2;
    d.nm = no * (no - 1) / 2;
    return d;
}

struct TensorMaps;  // TMA descriptors (emulated path), defined in emu_kernels.cu

}  // namespace ladder

struct ladder_plan_s {
    int no = 0, nv = 0, nchol = 0;
    int precision = LADDER_FP64;
    int nslices = ladder::kDefaultSlices;
    int device = 0;
    int num_sms = 0;
    int eri_clusters = 0;   // emulated ERI: CTA pairs that fit on the device at once
    int pair_clusters = 0;  // emulated ladder on CTA pairs: CTA pairs that fit at once
    size_t budget = 0;
    int n_a = 0, n_b = 0;
    int form = 0;  // emulated ladder form: 0 = plain (K = (c,d)), 1 = symmetric/antisymmetric
    int lad_bn = ladder::kEmuTileN;  // emulated ladder on one SM: pairs per column tile (16..96)
    int eri_chunk_max = 4;           // emulated ERI: longest exact K chunk, in blocks of 1024 (1..4)
    int pb = 0;                      // emulated: Cholesky vectors per slicing batch (0: all at once)
    int path = 0;     // 0: rebuild (ac|bd) per block pair; 1: factorised sum_P L_P T_ij L_P^T (FP64);
                      // 2: fused ERI -> ladder per block pair, no workspace (FP64)
    int fact_pb = 0;  // factorised path: Cholesky vectors per batch
    int shard_rank = 0, shard_world = 1;  // this plan holds shard `shard_rank` of `shard_world`
    std::vector<ladder::BlockPair> bps;
    int max_pairs = 0;
    ladder::WsLayout ws;
    // Host-buffer calls (ladder_apply_host): a copy stream and, per staging set, the events
    // "inputs copied" and "inputs free again"; created by the first such call.
    cudaStream_t h2d_stream = nullptr;
    cudaEvent_t host_ready[2] = {nullptr, nullptr};
    cudaEvent_t host_free[2] = {nullptr, nullptr};
    int host_parity = 0;
    // Device-side tables (allocated at plan time).
    void* d_tables = nullptr;          // pair lists (int2) + row_start tables (int)
    size_t tables_bytes = 0;
    unsigned* d_status = nullptr;      // status word
    unsigned long long wait_ns = ladder::kDefaultWaitNs;  // limit of the kernels' bounded waits
    double* d_partials = nullptr;      // energy reduction partials
    int n_partials = 0;
    // Optional per-kernel timing (benchmarks): event pairs tagged by kernel class.
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_kind;
    std::vector<int> ev_kernels;  // kernels launched between the two events of a slot
    size_t ev_used = 0;
    // Batched plans: sub-plans per instance, executed on worker streams forked from the
    // caller's stream (instance k runs on stream `stream_of[k]` with workspace slice
    // `ws_off[stream_of[k]]`).
    std::vector<ladder_plan_s*> sub;
    bool batched = false;
    int nstreams = 1;                  // worker streams used by the current schedule
    int max_streams = 1;               // streams the workspace is sized for
    std::vector<int> stream_of;        // per instance
    std::vector<int> order;            // execution order of instances
    std::vector<size_t> ws_off;        // per worker stream
    std::vector<cudaStream_t> workers;
    std::vector<cudaEvent_t> fork_join;  // [0] fork, [1 + w] join of worker w
    std::vector<double> model_s;       // modelled seconds per instance
    // Batched plans, grouped schedule (emulated path): the instances run in groups, each group
    // with one ERI launch and one ladder launch per ladder shape over all of its instances.
    int sched_groups = 0;                     // 0: worker-stream schedule; > 0: number of groups
    std::vector<std::vector<int>> groups;     // instances of each group
    std::vector<size_t> inst_off;             // workspace offset of each instance in the grouped schedule
    std::vector<size_t> group_eoff;           // first ERI entry (int4) of each group in d_group_entries
    std::vector<int> group_ecnt;              // ERI entries of each group
    void* d_group_entries = nullptr;
};

namespace ladder {

// Records an event pair around the `kernels` launches of one scope when the plan has
// timing enabled.
struct LaunchTimer {
    ladder_plan_s& p;
    cudaStream_t s;
    int kind;
    long slot = -1;
    LaunchTimer(const ladder_plan_s& plan, cudaStream_t stream, int k, int kernels = 1)
        : p(const_cast<ladder_plan_s&>(plan)), s(stream), kind(k) {
        if (p.timing && 2 * (p.ev_used + 1) <= p.ev_pool.size()) {
            slot = (long)p.ev_used++;
            p.ev_kind[slot] = kind;
            p.ev_kernels[slot] = kernels;
            cudaEventRecord(p.ev_pool[2 * slot], s);
        }
    }
    ~LaunchTimer() {
        if (slot >= 0) cudaEventRecord(p.ev_pool[2 * slot + 1], s);
    }
};

// fp64_kernels.cu
cudaError_t launch_fp64_block(const ladder_plan_s& p, const BlockPair& bp, const double* L,
                              const double* t2, double* R, void* ws, cudaStream_t s);
cudaError_t launch_fp64_factorised(const ladder_plan_s& p, const double* L, const double* t2, double* R, void* ws,
                                   cudaStream_t s);
// Fused ERI -> ladder kernel over the pairs of one block pair (no workspace); no^2 at most
// fused_fp64_max_rows().
cudaError_t launch_fp64_fused(const ladder_plan_s& p, const BlockPair& bp, const double* L, const double* t2,
                              double* R, cudaStream_t s);
int fused_fp64_max_rows();
// energy.cu
cudaError_t launch_energy(const ladder_plan_s& p, const double* t2, const double* R, double* E_dev,
                          cudaStream_t s);
// emu_kernels.cu
cudaError_t launch_emu_prep(const ladder_plan_s& p, const double* L, const double* t2, void* ws,
                            cudaStream_t s);
cudaError_t launch_emu_block(const ladder_plan_s& p, const BlockPair& bp, const double* L, double* R, void* ws,
                             cudaStream_t s);
// A group of emulated instances planned as one block pair each, run with one ERI launch and
// one ladder launch per ladder shape over all of them (ws[k]: instance k's workspace; entries:
// the group's ERI tiles with z = position of the instance in the group).
cudaError_t launch_emu_group(const ladder_plan_s& parent, const ladder_plan_s* const* subs, int n, void* const* ws,
                             const double* const* L, const double* const* t2, double* const* R, const int4* entries,
                             int nentries, cudaStream_t s);
int emu_max_group();  // most instances in one group
int emu_eri_stage_k(int nslices);  // K columns per pipeline stage of the emulated ERI
bool emu_supported(int no, int nv, int nchol, int nslices);
cudaError_t emu_set_attributes(int nslices);  // per device, before the first launch
// Co-resident clusters of the emulated CTA-pair kernels on the current device: kind 0 = ERI,
// kind 1 = ladder on CTA pairs.  0 if the query fails.
int emu_max_clusters(int nslices, int kind);

}  // namespace ladder
