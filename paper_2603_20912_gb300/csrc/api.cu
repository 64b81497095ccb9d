// Host runtime: the C ABI (include/ladder.h), the a/b block planner and the
// per-call orchestration.
//
// Planner (Sec. "An Asymmetric and Dynamic Splitting Protocol", Table 1, and
// the C-split loop nest): the paper sizes blocks along a, b (and c) so that
// the two consecutive contractions of one batch fit the free VRAM, with a and
// b split independently (n_a != n_b) and the budget taken as
// avail * 0.98 * 0.9.  Here L, t2 and R stay resident in HBM and only the
// intermediate of one (A, B) block pair -- the packed V block (a <= b only)
// and, on the emulated path, its digit slices and an int64 accumulator -- is
// staged in the workspace.  Among the (n_a, n_b) whose workspace fits the
// budget the planner picks the one with the lowest modelled time: per block
// pair, wave-quantised tile counts of the ERI GEMM and the ladder GEMM plus a
// fixed launch overhead.  The loop order over block pairs is the C-split
// order: b-blocks outer, a-blocks inner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ladder_internal.h"

using ladder::BlockPair;

namespace {

int map_cuda(cudaError_t e) { return e == cudaSuccess ? LADDER_OK : LADDER_ERR_CUDA; }

long long count_pairs(int a0, int a1, int b0, int b1) {
    long long n = 0;
    for (int a = a0; a < a1; ++a) n += std::max(0, b1 - std::max(a, b0));
    return n;
}

struct Geometry {
    int eri_tm, eri_tn, eri_occ;    // ERI tile and resident CTAs per SM
    int lad_tm, lad_tn, lad_occ;    // ladder tile
    double eri_tile_s;              // seconds for one ERI tile on one otherwise idle SM
    double lad_tile_s;              // seconds for one ladder tile
    double overhead_s;              // fixed cost per block pair
};

Geometry geometry_for(const ladder_plan_s& p) {
    Geometry g{};
    const double X = p.nchol, v2 = (double)p.nv * p.nv;
    if (p.precision == LADDER_FP64) {
        // FP64 DMMA: ~1.2 TFLOP/s per device; 64x64 tiles, several CTAs per SM.
        const double sm_rate = 1.2e12 / std::max(1, p.num_sms);
        g = {64, 64, 4, 64, 64, 4, 0, 0, 20e-6};
        g.eri_tile_s = 2.0 * 64 * 64 * X / sm_rate;
        g.lad_tile_s = 2.0 * 64 * 64 * v2 / sm_rate;
    } else {
        // BF16 tcgen05: ~1.5 PFLOP/s sustained; S(S+1)/2 slice products per element.
        const double pairs = 0.5 * p.nslices * (p.nslices + 1);
        const double sm_rate = 1.5e15 / std::max(1, p.num_sms);
        // ladder tiles: 96 pairs x (i,j) rows of 128 (one SM) or 256 (CTA pair)
        const int lrows = p.no * p.no <= 128 ? 128 : 256;
        g = {256, ladder::kEmuTileN, 1, ladder::kEmuTileN, lrows, 1, 0, 0, 25e-6};
        g.eri_tile_s = 2.0 * 128 * ladder::kEmuTileN * X * pairs / sm_rate + 3e-6;  // per SM of the pair
        g.lad_tile_s = 2.0 * ladder::kEmuTileN * lrows * v2 * pairs / sm_rate / (lrows / 128) + 3e-6;
    }
    return g;
}

long long count_eri_tiles(const BlockPair& bp, int nv, int tm, int tn) {
    const int na = bp.a1 - bp.a0, nb = bp.b1 - bp.b0;
    const long long M = (long long)na * nv, N = (long long)nb * nv;
    const long long nrt = (M + tm - 1) / tm, nqt = (N + tn - 1) / tn;
    long long tiles = 0;
    for (long long rt = 0; rt < nrt; ++rt) {
        const int a_min = bp.a0 + (int)(rt * tm / nv);
        // smallest qt whose largest b reaches a_min
        long long lo = 0, hi = nqt;
        while (lo < hi) {
            const long long mid = (lo + hi) / 2;
            const long long last = std::min((mid + 1) * tn, N) - 1;
            const int b_max = bp.b0 + (int)(last / nv);
            if (b_max >= a_min) hi = mid; else lo = mid + 1;
        }
        tiles += nqt - lo;
    }
    return tiles;
}

std::vector<BlockPair> enumerate_blocks(int nv, int na, int nb) {
    std::vector<BlockPair> out;
    for (int b0 = 0; b0 < nv; b0 += nb) {          // C-split order: b outer, a inner
        const int b1 = std::min(nv, b0 + nb);
        for (int a0 = 0; a0 < nv; a0 += na) {
            const int a1 = std::min(nv, a0 + na);
            const long long n = count_pairs(a0, a1, b0, b1);
            if (n > 0) out.push_back(BlockPair{a0, a1, b0, b1, (int)n, 0, 0});
        }
    }
    return out;
}

int apply_blocking(ladder_plan_s& p, int na, int nb);

ladder::WsLayout layout_for(const ladder_plan_s& p, long long max_pairs) {
    using ladder::align_up;
    using ladder::kAlign;
    ladder::WsLayout w;
    const size_t nv2 = (size_t)p.nv * p.nv, no2 = (size_t)p.no * p.no;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off = align_up(off + bytes, kAlign); return o; };
    if (p.path == 1) {
        const size_t npij = (size_t)p.no * (p.no + 1) / 2;
        w.w_blk = take(npij * nv2 * (size_t)p.fact_pb * sizeof(double));
    } else if (p.path == 2) {
        // fused path: (ac|bd) stays on the chip, no workspace
    } else if (p.precision == LADDER_FP64) {
        w.v_blk = take((size_t)max_pairs * nv2 * sizeof(double));
    } else {
        // (c, d) rows padded to vp (ladder::emu_vp): K index c*vp + d, zero for d >= nv.
        const size_t S = p.nslices;
        const size_t vp = (size_t)ladder::emu_vp(p.nv), nvp = (size_t)p.nv * vp;
        const size_t batch = p.pb > 0 && p.pb < p.nchol ? (size_t)p.pb : (size_t)p.nchol;
        const size_t kpad = nvp, xpad = align_up(batch, 8);
        const size_t G = ladder::kExpGroupRows;
        // V digit planes, or V as int64 for the symmetric/antisymmetric form (combined first)
        w.v_blk = take((p.form == 0 ? S * 2 : 8) * (size_t)max_pairs * kpad);
        w.lt_slices = take(S * nvp * xpad * 2);
        w.lt_exp = take(((nvp + G - 1) / G) * 4);
        if (p.form == 0) {
            w.rp_int = take((size_t)max_pairs * no2 * 8);
            w.t_slices = take(S * no2 * kpad * 2);
            w.t_gmax = take(((no2 + G - 1) / G) * 8);
            w.t_exp = take(((no2 + G - 1) / G) * 4);
        } else {
            const ladder::PmDims d = ladder::pm_dims(p.no, p.nv);
            w.vp_blk = take(S * (size_t)max_pairs * d.kp_pad * 2);
            w.vm_blk = take(S * (size_t)max_pairs * d.km_pad * 2);
            w.tp_slices = take(S * (size_t)d.np * d.kp_pad * 2);
            w.tm_slices = take(S * (size_t)d.nm * d.km_pad * 2);
            w.tp_gmax = take(((d.np + G - 1) / G) * 8);
            w.tm_gmax = take(((d.nm + G - 1) / G) * 8);
            w.tp_exp = take(((d.np + G - 1) / G) * 4);
            w.tm_exp = take(((d.nm + G - 1) / G) * 4);
            w.rpx = take((size_t)max_pairs * d.np * 8);
            w.rpy = take((size_t)max_pairs * d.nm * 8);
        }
        w.v_exp = take(nv2 * 4);
        w.lnorm = take((size_t)p.nv * 8);
        w.lsq = take(nv2 * 8);
        const size_t nblk = (xpad + ladder::kEmuChunkK - 1) / ladder::kEmuChunkK;
        w.lt_norm2 = take(S * nvp * nblk * 4);
        w.eri_cand = take(S * 3 * 4);
        w.eri_kbc = take(4);
    }
    w.total = std::max<size_t>(off, kAlign);
    return w;
}

long long max_pairs_of(const std::vector<BlockPair>& bps) {
    long long m = 0;
    for (auto& b : bps) m = std::max<long long>(m, b.npairs);
    return m;
}

// Number of ERI entries (tiles) eri_entries keeps for one block pair, from the row segments and
// the column-tile rule directly: segment by segment, 32 chunks to a tile, a tile with smallest
// key k meeting the column tiles whose last b reaches k (no chunk list is built).
long long eri_tile_count(const BlockPair& bp, int nv, int tile_n) {
    const int vp = ladder::emu_vp(nv), cr = 8;
    const long long N = (long long)(bp.b1 - bp.b0) * vp, nqt = (N + tile_n - 1) / tile_n;
    auto cols = [&](int key) -> long long {   // column tiles holding a b >= key
        const long long first = (long long)std::max(0, key - bp.b0) * vp;
        return first >= N ? 0 : nqt - first / tile_n;
    };
    long long total = 0;
    int in_tile = 0, kmin = nv;
    // m chunks with keys key0, key0 + step, ... (ascending within the segment)
    auto segment = [&](long long m, int key0, int step) {
        for (long long j = 0; j < m;) {
            const long long take = std::min<long long>(m - j, 32 - in_tile);
            kmin = std::min(kmin, key0 + step * (int)j);
            in_tile += (int)take;
            j += take;
            if (in_tile == 32) {
                total += cols(kmin);
                in_tile = 0;
                kmin = nv;
            }
        }
    };
    for (int x = bp.a0; x < bp.a1; ++x) segment((nv - x + cr - 1) / cr, x, 0);
    for (int x = 0; x < bp.a0; ++x) segment((bp.a1 - bp.a0 + cr - 1) / cr, bp.a0, cr);
    if (in_tile > 0) total += cols(kmin);
    return total;
}

double model_time(const ladder_plan_s& p, const std::vector<BlockPair>& bps) {
    const Geometry g = geometry_for(p);
    const double slots_e = (double)p.num_sms * g.eri_occ, slots_l = (double)p.num_sms * g.lad_occ;
    const long long nt = (long long)(p.no * p.no + g.lad_tn - 1) / g.lad_tn;
    double t = 0.0;
    for (auto& bp : bps) {
        const long long te = p.precision == LADDER_FP64 ? count_eri_tiles(bp, p.nv, g.eri_tm, g.eri_tn)
                                                        : eri_tile_count(bp, p.nv, g.eri_tn);
        const long long tl = ((long long)(bp.npairs + g.lad_tm - 1) / g.lad_tm) * nt;
        t += std::ceil(te / (p.precision == LADDER_FP64 ? slots_e : slots_e / 2)) * g.eri_occ * g.eri_tile_s;
        t += std::ceil(tl / slots_l) * g.lad_occ * g.lad_tile_s;
        t += g.overhead_s;
    }
    return t;
}

// Evaluation order (Sec. "Acceleration of CC calculations"): rebuilding (ac|bd) costs
// 2 X v^2 p + 2 o^2 v^2 p flops with the a <= b packing; the factorised order
// R_ij = sum_P L_P T_ij L_P^T costs 4 X v^3 per amplitude pair, o(o+1)/2 pairs with i <= j.
// Both run on the same FP64 DMMA tiles, so the flop counts compare directly; the factorised
// order is taken when it needs 1.25x fewer flops (it streams a W batch through HBM per
// Cholesky batch).  Otherwise an FP64 plan takes the rebuild order fused on the chip (path 2:
// the same flops, no V round trip through HBM and no workspace, measured faster than the
// unfused rebuild at every shape it was timed on) when its accumulators hold the no^2
// amplitude rows.  The emulated path has only the rebuild order through HBM.
double eri_path_flops(int no, int nv, int nchol) {
    const double p = 0.5 * (double)nv * (nv + 1), v2 = (double)nv * nv;
    return 2.0 * nchol * v2 * p + 2.0 * (double)no * no * v2 * p;
}
double fact_path_flops(int no, int nv, int nchol) {
    return 4.0 * nchol * (0.5 * no * (no + 1.0)) * (double)nv * nv * nv;
}
int auto_path(int no, int nv, int nchol, int precision) {
    if (precision != LADDER_FP64) return 0;
    if (1.25 * fact_path_flops(no, nv, nchol) < eri_path_flops(no, nv, nchol)) return 1;
    return (long long)no * no <= ladder::fused_fp64_max_rows() ? 2 : 0;
}

// Cholesky vectors per batch of the factorised path: as many as the budget holds (W is
// 8 o(o+1)/2 nv^2 bytes per vector), at most nchol and at most 65535 / (o(o+1)/2) (grid z of the
// first GEMM); LADDER_ERR_BUDGET when not even one vector fits.
int use_factorised(ladder_plan_s& p) {
    const long long npij = (long long)p.no * (p.no + 1) / 2;
    const double per = 8.0 * npij * (double)p.nv * p.nv;
    long long pb = (long long)std::floor((double)p.budget / per);
    pb = std::min<long long>(pb, p.nchol);
    pb = std::min<long long>(pb, 65535 / npij);
    if (pb < 1) return LADDER_ERR_BUDGET;
    const int old_pb = p.fact_pb, old_path = p.path;
    p.fact_pb = (int)pb;
    p.path = 1;
    const ladder::WsLayout w = layout_for(p, 0);
    if (w.total > p.budget) {
        p.fact_pb = old_pb;
        p.path = old_path;
        return LADDER_ERR_BUDGET;
    }
    p.ws = w;
    return LADDER_OK;
}

// Fused path (FP64): the plan's block pairs -- one block pair of all pairs unless the plan is a
// shard -- walked by the fused ERI -> ladder kernel, which needs no workspace; its accumulators
// hold no^2 <= fused_fp64_max_rows() amplitude rows (LADDER_ERR_UNSUPPORTED otherwise).
int use_fused(ladder_plan_s& p) {
    if (p.precision != LADDER_FP64 || (long long)p.no * p.no > ladder::fused_fp64_max_rows())
        return LADDER_ERR_UNSUPPORTED;
    const int old_path = p.path;
    p.path = 2;
    if (p.shard_world > 1) {
        p.ws = layout_for(p, p.max_pairs);
        return LADDER_OK;
    }
    const int rc = apply_blocking(p, p.nv, p.nv);
    if (rc != LADDER_OK) {
        p.path = old_path;
        p.ws = layout_for(p, old_path == 1 ? 0 : p.max_pairs);
    }
    return rc;
}

// Modelled seconds of one call (scheduling of batched plans).
double plan_time(const ladder_plan_s& p) {
    if (p.path == 1) return fact_path_flops(p.no, p.nv, p.nchol) / 1.0e12 + 20e-6;
    return model_time(p, p.bps);
}

// ERI row tiles of the emulated path.  The rows of L^T are (x, y) = x vp + y, and L^P is
// symmetric, so the rows (x, y) and (y, x) hold the same vector: only rows with x <= y are
// multiplied.  A computed row (x, y) serves the V rows (x, b) at column block y (x in the block's
// a range, b >= x) and (y, b) at column block x (y in the a range, x < y, b >= y).  The rows one
// block needs are the segments (x, [x, nv)) for x in [a0, a1) and (x, [a0, a1)) for x < a0; each
// is cut into chunks of 8 consecutive rows (one TMA box), 32 chunks to a 256-row tile, the last
// tile padded with empty chunks.  key[t]: the smallest b that a row of tile t stores to.
struct EriRowTiles {
    std::vector<int> chunks;  // (first row, rows) per chunk
    std::vector<int> key;     // per tile
};

EriRowTiles eri_row_tiles(const BlockPair& bp, int nv) {
    const int vp = ladder::emu_vp(nv), cr = ladder::kEmuTile * 2 / 32;   // 8 rows per chunk
    EriRowTiles t;
    std::vector<int> ckey;
    auto segment = [&](int x, int y0, int y1, bool upper) {
        for (int y = y0; y < y1; y += cr) {
            t.chunks.push_back(x * vp + y);
            t.chunks.push_back(std::min(cr, y1 - y));
            ckey.push_back(upper ? x : y);
        }
    };
    for (int x = bp.a0; x < bp.a1; ++x) segment(x, x, nv, true);
    for (int x = 0; x < bp.a0; ++x) segment(x, bp.a0, bp.a1, false);
    const size_t ntile = (ckey.size() + 31) / 32;
    t.chunks.resize(2 * 32 * ntile, 0);
    t.key.assign(ntile, nv);
    for (size_t c = 0; c < ckey.size(); ++c) t.key[c / 32] = std::min(t.key[c / 32], ckey[c]);
    return t;
}

// Build device tables for the chosen blocking: per block pair its pair list
// (int2 (a, b), a-major) and row_start (first packed row of each a).
// ERI work entries of one block pair, (rt, qt, 0, 0): a 256-row tile rt (computed by a CTA pair,
// 128 rows each) and a 96-column tile qt of (b,d), kept when one of its rows stores to one of
// its b.  Order: a band of row tiles whose operand slices take ~16 MB of L2 stays resident while
// every column tile of the band streams past it (at no=20 nv=400 nchol=1260 bands of 16, 40 and
// 120 MB all took the same time; the smallest moved the fewest bytes from DRAM).
std::vector<int> eri_entries(const BlockPair& bp, int nv, int tile_n, size_t row_bytes) {
    const EriRowTiles rt = eri_row_tiles(bp, nv);
    nv = ladder::emu_vp(nv);  // columns run over the padded (b, d) range
    std::vector<int> out;
    const long long N = (long long)(bp.b1 - bp.b0) * nv;
    const int nrt = (int)rt.key.size(), nqt = (int)((N + tile_n - 1) / tile_n);
    const int band = (int)std::max<size_t>(4, std::min<size_t>(32, (16u << 20) / std::max<size_t>(1, row_bytes * 256)));
    for (int r0 = 0; r0 < nrt; r0 += band)
        for (int qt = 0; qt < nqt; ++qt)
            for (int r = r0; r < std::min(nrt, r0 + band); ++r) {
                const long long last = std::min((long long)(qt + 1) * tile_n, N) - 1;
                if (rt.key[r] > bp.b0 + (int)(last / nv)) continue;
                out.push_back(r);
                out.push_back(qt);
                out.push_back(0);
                out.push_back(0);
            }
    return out;
}

int build_tables(ladder_plan_s& p) {
    size_t n_int2 = 0, n_int = 0;
    std::vector<std::vector<int>> tiles, chunks;
    for (auto& bp : p.bps) n_int2 += bp.npairs;
    if (p.precision != LADDER_FP64)
        for (auto& bp : p.bps) {
            tiles.push_back(eri_entries(bp, p.nv, ladder::kEmuTileN,
                                        (size_t)p.nslices * 2 * ladder::align_up((size_t)p.nchol, 8)));
            chunks.push_back(eri_row_tiles(bp, p.nv).chunks);
            n_int2 += tiles.back().size() / 2 + chunks.back().size() / 2;
        }
    n_int2 += 1;  // room to align the int4 ERI entries to 16 bytes
    for (auto& bp : p.bps) n_int += (size_t)(bp.a1 - bp.a0 + 1);
    std::vector<int> host(2 * n_int2 + n_int);
    size_t o2 = 0, oi = 2 * n_int2;
    for (auto& bp : p.bps) {
        bp.pairs_off = o2;
        bp.rows_off = oi;
        int row = 0;
        for (int a = bp.a0; a < bp.a1; ++a) {
            host[oi++] = row;
            for (int b = std::max(a, bp.b0); b < bp.b1; ++b) {
                host[2 * o2] = a;
                host[2 * o2 + 1] = b;
                ++o2;
                ++row;
            }
        }
        host[oi++] = row;
    }
    o2 += o2 & 1;  // int4 entries start on a 16-byte boundary
    for (size_t k = 0; k < tiles.size(); ++k) {
        p.bps[k].tiles_off = o2;                       // in int2 units; entries are int4 = 2 int2
        p.bps[k].ntiles = (int)(tiles[k].size() / 4);  // number of entries
        for (size_t t = 0; t < tiles[k].size(); ++t) host[2 * o2 + t] = tiles[k][t];
        o2 += tiles[k].size() / 2;
        p.bps[k].chunks_off = o2;
        for (size_t t = 0; t < chunks[k].size(); ++t) host[2 * o2 + t] = chunks[k][t];
        o2 += chunks[k].size() / 2;
    }
    if (p.d_tables) {
        cudaFree(p.d_tables);
        p.d_tables = nullptr;
    }
    p.tables_bytes = std::max<size_t>(host.size() * sizeof(int), 16);
    if (cudaMalloc(&p.d_tables, p.tables_bytes) != cudaSuccess) return LADDER_ERR_CUDA;
    if (!host.empty() &&
        cudaMemcpy(p.d_tables, host.data(), host.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
        return LADDER_ERR_CUDA;
    return LADDER_OK;
}

int apply_blocking(ladder_plan_s& p, int na, int nb) {
    std::vector<BlockPair> bps = enumerate_blocks(p.nv, na, nb);
    const ladder::WsLayout w = layout_for(p, max_pairs_of(bps));
    if (w.total > p.budget) return LADDER_ERR_BUDGET;
    p.n_a = na;
    p.n_b = nb;
    p.bps = std::move(bps);
    p.max_pairs = (int)max_pairs_of(p.bps);
    p.ws = w;
    return build_tables(p);
}

// Owner of each block pair when the pairs are spread over `world` ranks: largest pair
// count first (ties by position), each to the least-loaded rank (ties: the lower rank).
// Pure host arithmetic, so every rank computes the same partition.
std::vector<int> shard_owner(const std::vector<long long>& npairs, int world) {
    const int n = (int)npairs.size();
    std::vector<int> order(n), owner(n, 0);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return npairs[x] > npairs[y]; });
    std::vector<long long> load(world, 0);
    for (int i : order) {
        const int r = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        owner[i] = r;
        load[r] += npairs[i];
    }
    return owner;
}

int select_blocking(const ladder_plan_s& p, int* out_na, int* out_nb, int min_block_pairs = 1) {
    std::vector<int> cand;
    for (int k = 1; k <= p.nv; ++k) {
        const int n = (p.nv + k - 1) / k;
        if (cand.empty() || cand.back() != n) cand.push_back(n);
    }
    // Candidate (n_a, n_b) ordered by the number of block pairs: the model time
    // grows with it, so the best feasible blocking is among the first feasible ones.
    struct Combo { double nbp; int na, nb; };
    std::vector<Combo> combos;
    for (int na : cand)
        for (int nb : cand) combos.push_back({std::ceil((double)p.nv / na) * std::ceil((double)p.nv / nb), na, nb});
    std::stable_sort(combos.begin(), combos.end(), [](const Combo& x, const Combo& y) { return x.nbp < y.nbp; });
    double best = 1e300;
    int bna = 0, bnb = 0, evaluated = 0;
    for (const Combo& c : combos) {
        std::vector<BlockPair> bps = enumerate_blocks(p.nv, c.na, c.nb);
        if ((int)bps.size() < min_block_pairs) continue;
        if (layout_for(p, max_pairs_of(bps)).total > p.budget) continue;
        const double t = model_time(p, bps);
        if (t < best * (1 - 1e-9)) {
            best = t;
            bna = c.na;
            bnb = c.nb;
        }
        if (++evaluated >= 64) break;
    }
    if (bna == 0) return LADDER_ERR_BUDGET;
    *out_na = bna;
    *out_nb = bnb;
    return LADDER_OK;
}

// The block pairs rank `rank` of `world` owns: the plan's blocking, or, when it has fewer than
// 2 * world block pairs and the shape allows more, the best blocking under the same budget with
// at least that many; then the longest-first partition of shard_owner.
int shard_select(const ladder_plan_s& p, int rank, int world, int* na, int* nb, std::vector<BlockPair>* mine) {
    const long long most = (long long)p.nv * (p.nv + 1) / 2;
    const int want = (int)std::min<long long>(2LL * world, most);
    std::vector<BlockPair> bps = p.bps;
    *na = p.n_a;
    *nb = p.n_b;
    if ((int)bps.size() < want) {
        const int rc = select_blocking(p, na, nb, want);
        if (rc != LADDER_OK) return rc;
        bps = enumerate_blocks(p.nv, *na, *nb);
    }
    std::vector<long long> np;
    for (auto& b : bps) np.push_back(b.npairs);
    const std::vector<int> owner = shard_owner(np, world);
    mine->clear();
    for (size_t i = 0; i < bps.size(); ++i)
        if (owner[i] == rank) mine->push_back(bps[i]);
    return LADDER_OK;
}

int choose_blocking(ladder_plan_s& p) {
    int na = 0, nb = 0;
    const int rc = select_blocking(p, &na, &nb);
    if (rc != LADDER_OK) return rc;
    return apply_blocking(p, na, nb);
}

// Modelled extra time of slicing the Cholesky vectors in batches: every block pair re-slices all
// of L (reads 8 and writes 2S bytes per element at ~3 TB/s) and launches three more kernels per
// batch, and every ERI tile drains its accumulators once more per batch.
double pbatch_overhead(const ladder_plan_s& p, const std::vector<BlockPair>& bps) {
    if (p.pb <= 0 || p.pb >= p.nchol) return 0.0;
    const double rows = (double)p.nv * ladder::emu_vp(p.nv);
    const int nbat = (p.nchol + p.pb - 1) / p.pb;
    const double slice = rows * p.nchol * (8.0 + 2.0 * p.nslices) / 3.0e12;
    double tiles = 0.0;
    for (auto& bp : bps) tiles += (double)eri_tile_count(bp, p.nv, ladder::kEmuTileN);
    const double clusters = std::max(1, p.num_sms / 2);
    return bps.size() * (slice + nbat * 30e-6) + tiles / clusters * (nbat - 1) * 4e-6;
}

// Emulated path: whether to slice the Cholesky vectors a batch at a time (the L^T digit planes of
// all vectors take 2S bytes per element of L, which at large nchol leaves little of the budget
// for V blocks).  Batches need the split form's int64 V, which adds the exact sums of the batches.
// Candidates: all vectors at once (the blocking the plan holds, if `have`) and batches of 8192,
// 4096, 2048 and 1024 vectors; the lowest modelled time wins (a batch must win by 3 %).  Host only:
// returns the chosen batch (0: none) and, for a batch, its blocking; leaves the plan as it was.
int select_pbatch(ladder_plan_s& p, bool have, int* out_na, int* out_nb) {
    if (p.precision == LADDER_FP64 || p.nchol <= 1024) return 0;
    double best = have ? model_time(p, p.bps) : 1e300;
    int best_pb = 0;
    const int pb0 = p.pb, form0 = p.form;
    for (int pb : {8192, 4096, 2048, 1024}) {
        if (pb >= p.nchol) continue;
        p.pb = pb;
        p.form = 1;
        int na = 0, nb = 0;
        if (select_blocking(p, &na, &nb) == LADDER_OK) {
            const std::vector<BlockPair> bps = enumerate_blocks(p.nv, na, nb);
            const double t = model_time(p, bps) + pbatch_overhead(p, bps);
            if (t < best * 0.97) {
                best = t;
                best_pb = pb;
                *out_na = na;
                *out_nb = nb;
            }
        }
    }
    p.pb = pb0;
    p.form = form0;
    return best_pb;
}

bool aligned256(const void* ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 255u) == 0; }

void free_events(ladder_plan_s* p) {
    for (auto e : p->ev_pool) cudaEventDestroy(e);
    p->ev_pool.clear();
    p->ev_kind.clear();
    p->ev_kernels.clear();
    p->ev_used = 0;
    p->timing = false;
}

void destroy_plan(ladder_plan_s* p) {
    if (!p) return;
    for (auto* s : p->sub) destroy_plan(s);
    for (auto w : p->workers) cudaStreamDestroy(w);
    for (auto e : p->fork_join) cudaEventDestroy(e);
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    free_events(p);
    if (p->h2d_stream) cudaStreamDestroy(p->h2d_stream);
    for (int s = 0; s < 2; ++s) {
        if (p->host_ready[s]) cudaEventDestroy(p->host_ready[s]);
        if (p->host_free[s]) cudaEventDestroy(p->host_free[s]);
    }
    if (p->d_tables) cudaFree(p->d_tables);
    if (p->d_status) cudaFree(p->d_status);
    if (p->d_partials) cudaFree(p->d_partials);
    if (p->d_group_entries) cudaFree(p->d_group_entries);
    if (cur >= 0 && cur != p->device) cudaSetDevice(cur);
    delete p;
}

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Emulated ladder form from a cost model of a whole call over all a <= b pairs: the ERI (the same
// in both forms; K = nchol, symmetric rows), the ladder GEMM, whose MMA rows are padded to its tiles (128 rows
// on one SM up to 128 (i,j) rows, else 256 on CTA pairs) and which the symmetric/antisymmetric
// form halves in K and splits into rows i <= j and i < j, and the split's one pass that reads V
// as int64 and writes the V' and V'' digit planes (~3.5 TB/s measured).  The split is chosen
// when the model gives the call a 5 % lead.
int auto_form(int no, int nv, int nchol, int nslices) {
    const double pairs = 0.5 * nv * (nv + 1.0);
    auto rows_pad = [](double r) { return r <= ladder::kEmuTile ? ladder::kEmuTile : std::ceil(r / 256.0) * 256.0; };
    const double vp = ladder::emu_vp(nv);
    const double per_row_k = pairs * 2.0 * nslices * (nslices + 1) / 2 / 1.3e15;   // s per (row, K element)
    // the ERI multiplies the rows x <= y of L^T against the columns b >= x: (2 nv + 1) / (3 nv)
    // of the a <= b pairs' row-column products
    const double eri = (double)nchol * nv * vp * per_row_k * (2.0 * nv + 1.0) / (3.0 * nv);
    const double plain = eri + rows_pad((double)no * no) * nv * vp * per_row_k;
    const ladder::PmDims d = ladder::pm_dims(no, nv);
    double pm = eri + rows_pad(d.np) * (double)d.kp * per_row_k;
    if (d.nm > 0) pm += rows_pad(d.nm) * (double)d.km * per_row_k;
    pm += (8.0 + 2.0 * nslices) * pairs * nv * vp / 3.5e12;   // read int64 V, write V' and V''
    return pm < 0.95 * plain ? 1 : 0;
}

// split_ok = false keeps the plain form.
int make_plan(ladder_plan_s** out, int no, int nv, int nchol, int precision, int nslices, size_t budget,
              int device, bool split_ok = true, bool pbatch_ok = true) {
    *out = nullptr;
    if (no < 1 || nv < 1 || nchol < 1) return LADDER_ERR_ARG;
    if ((long long)no * no > (1 << 20) || nv > 4096) return LADDER_ERR_ARG;
    if (precision == LADDER_EMU_INT8) return LADDER_ERR_UNSUPPORTED;
    if (precision != LADDER_FP64 && precision != LADDER_EMU_BF16) return LADDER_ERR_ARG;
    if (nslices == 0) nslices = ladder::kDefaultSlices;
    if (precision == LADDER_EMU_BF16) {
        if (nslices < 5 || nslices > 8) return LADDER_ERR_ARG;
        if (!ladder::emu_supported(no, nv, nchol, nslices)) return LADDER_ERR_UNSUPPORTED;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) return LADDER_ERR_CUDA;
    if (device < 0 || device >= ndev) return LADDER_ERR_ARG;
    DeviceGuard guard(device);
    if (!guard.ok) return LADDER_ERR_CUDA;
    auto* p = new (std::nothrow) ladder_plan_s();
    if (!p) return LADDER_ERR_CUDA;
    p->no = no;
    p->nv = nv;
    p->nchol = nchol;
    p->precision = precision;
    p->nslices = precision == LADDER_FP64 ? 0 : nslices;
    p->device = device;
    if (cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        destroy_plan(p);
        return LADDER_ERR_CUDA;
    }
    if (budget == 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            destroy_plan(p);
            return LADDER_ERR_CUDA;
        }
        budget = (size_t)((double)free_b * 0.98 * 0.9);
    }
    p->budget = budget;
    if (precision != LADDER_FP64) {
        if (ladder::emu_set_attributes(nslices) != cudaSuccess) {
            destroy_plan(p);
            return LADDER_ERR_CUDA;
        }
        p->eri_clusters = ladder::emu_max_clusters(nslices, 0);
        p->pair_clusters = ladder::emu_max_clusters(nslices, 1);
    }
    p->form = precision == LADDER_FP64 || !split_ok ? 0 : auto_form(no, nv, nchol, p->nslices);
    int rc = choose_blocking(*p);
    if (rc == LADDER_ERR_BUDGET && p->form == 1) {   // the split needs more workspace: fall back
        p->form = 0;
        rc = choose_blocking(*p);
    }
    // Emulated: slicing the Cholesky vectors in batches when that lets larger blocks fit (or any).
    if ((rc == LADDER_OK || rc == LADDER_ERR_BUDGET) && precision != LADDER_FP64 && pbatch_ok) {
        int na = 0, nb = 0;
        const int pb = select_pbatch(*p, rc == LADDER_OK, &na, &nb);
        if (pb > 0) {
            p->pb = pb;
            p->form = 1;
            rc = apply_blocking(*p, na, nb);
        }
    }
    // FP64: the factorised order when the model prefers it and its batch fits (also when no
    // blocking of the rebuild order fits the budget).
    if ((rc == LADDER_OK || rc == LADDER_ERR_BUDGET) && precision == LADDER_FP64 &&
        (auto_path(no, nv, nchol, precision) == 1 || rc == LADDER_ERR_BUDGET)) {
        if (use_factorised(*p) == LADDER_OK) rc = LADDER_OK;
    }
    // FP64: the fused path when the model prefers it, or when nothing else fits (it needs no
    // workspace).
    if ((rc == LADDER_OK || rc == LADDER_ERR_BUDGET) && precision == LADDER_FP64 &&
        (auto_path(no, nv, nchol, precision) == 2 || rc == LADDER_ERR_BUDGET)) {
        if (use_fused(*p) == LADDER_OK) rc = LADDER_OK;
    }
    if (rc == LADDER_OK) {
        if (cudaMalloc(&p->d_status, sizeof(unsigned)) != cudaSuccess ||
            cudaMemset(p->d_status, 0, sizeof(unsigned)) != cudaSuccess)
            rc = LADDER_ERR_CUDA;
    }
    if (rc == LADDER_OK) {
        const long long ntile = (nv + 31) / 32;
        const long long units = (long long)no * no * ntile * ntile;
        p->n_partials = (int)std::max<long long>(1, std::min<long long>(units, 4LL * p->num_sms));
        if (cudaMalloc(&p->d_partials, sizeof(double) * (p->n_partials + 1)) != cudaSuccess) rc = LADDER_ERR_CUDA;
    }
    if (rc != LADDER_OK) {
        destroy_plan(p);
        return rc;
    }
    *out = p;
    return LADDER_OK;
}

// Longest-processing-time-first assignment of instances to k worker streams; the
// workspace of a stream is the largest workspace among its instances.
void schedule_batched(ladder_plan_s& p, int k) {
    p.sched_groups = 0;
    const int n = (int)p.sub.size();
    k = std::max(1, std::min(k, std::min(n, p.max_streams)));
    p.nstreams = k;
    p.order.resize(n);
    for (int i = 0; i < n; ++i) p.order[i] = i;
    std::stable_sort(p.order.begin(), p.order.end(), [&](int x, int y) { return p.model_s[x] > p.model_s[y]; });
    std::vector<double> load(k, 0.0);
    p.stream_of.assign(n, 0);
    for (int i : p.order) {
        const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        p.stream_of[i] = w;
        load[w] += p.model_s[i];
    }
}

// An instance can join a group when it runs on the emulated path as a single block pair and slices
// all its Cholesky vectors at once.
bool groupable(const ladder_plan_s& s) {
    return s.precision != LADDER_FP64 && s.bps.size() == 1 && (s.pb <= 0 || s.pb >= s.nchol);
}

// Ladder items an instance adds to its group's launches: one in the plain form; X, and Y when
// there are rows i < j and pairs c < d, in the split form.
int ladder_items_of(const ladder_plan_s& s) { return s.form == 1 && s.no > 1 && s.nv > 1 ? 2 : 1; }

// Grouped schedule: first-fit decreasing of the instances' workspaces into groups of at most
// `cap` bytes, emu_max_group() instances and emu_max_group() ladder items (an instance that cannot
// be grouped runs alone),
// and the device list of every group's ERI tiles with z = position of the instance in its group.
int schedule_groups(ladder_plan_s& p, size_t cap) {
    const int n = (int)p.sub.size();
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return p.sub[x]->ws.total > p.sub[y]->ws.total; });
    std::vector<std::vector<int>> groups;
    std::vector<size_t> used;
    std::vector<int> items;
    p.inst_off.assign(n, 0);
    for (int k : order) {
        const size_t need = ladder::align_up(p.sub[k]->ws.total, ladder::kAlign);
        if (need > p.ws.total) return LADDER_ERR_BUDGET;
        int g = -1;
        if (groupable(*p.sub[k]))
            for (int j = 0; j < (int)groups.size() && g < 0; ++j)
                if (groupable(*p.sub[groups[j][0]]) && used[j] + need <= cap &&
                    (int)groups[j].size() < ladder::emu_max_group() &&
                    items[j] + ladder_items_of(*p.sub[k]) <= ladder::emu_max_group())
                    g = j;
        if (g < 0) {
            groups.push_back({});
            used.push_back(0);
            items.push_back(0);
            g = (int)groups.size() - 1;
        }
        p.inst_off[k] = used[g];
        used[g] += need;
        items[g] += ladder_items_of(*p.sub[k]);
        groups[g].push_back(k);
    }
    std::vector<int> host;
    p.group_eoff.clear();
    p.group_ecnt.clear();
    for (auto& grp : groups) {
        p.group_eoff.push_back(host.size() / 4);
        int cnt = 0;
        if (grp.size() > 1 || groupable(*p.sub[grp[0]]))
            for (int i = 0; i < (int)grp.size(); ++i) {
                const ladder_plan_s& q = *p.sub[grp[i]];
                const std::vector<int> t = eri_entries(q.bps[0], q.nv, ladder::kEmuTileN,
                                                       (size_t)q.nslices * 2 * ladder::align_up((size_t)q.nchol, 8));
                for (size_t j = 0; j < t.size(); j += 4) {
                    host.push_back(t[j]);
                    host.push_back(t[j + 1]);
                    host.push_back(i);
                    host.push_back(0);
                    ++cnt;
                }
            }
        p.group_ecnt.push_back(cnt);
    }
    if (p.d_group_entries) {
        cudaFree(p.d_group_entries);
        p.d_group_entries = nullptr;
    }
    if (cudaMalloc(&p.d_group_entries, std::max<size_t>(16, host.size() * sizeof(int))) != cudaSuccess)
        return LADDER_ERR_CUDA;
    if (!host.empty() &&
        cudaMemcpy(p.d_group_entries, host.data(), host.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
        return LADDER_ERR_CUDA;
    p.groups = std::move(groups);
    p.sched_groups = (int)p.groups.size();
    return LADDER_OK;
}

}  // namespace

extern "C" {

int ladder_plan(ladder_plan_t* out, int no, int nv, int nchol, int precision, int nslices,
                size_t ws_budget_bytes, int device) {
    if (!out) return LADDER_ERR_ARG;
    return make_plan(out, no, nv, nchol, precision, nslices, ws_budget_bytes, device);
}

int ladder_plan_set_blocks(ladder_plan_t plan, int n_a, int n_b) {
    if (!plan || plan->batched || plan->shard_world > 1) return LADDER_ERR_ARG;
    if (n_a < 1 || n_b < 1 || n_a > plan->nv || n_b > plan->nv) return LADDER_ERR_ARG;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return LADDER_ERR_CUDA;
    // Validate before touching the plan so a rejected request leaves it intact.  A blocking
    // belongs to the rebuild order: a factorised plan returns to it.
    std::vector<BlockPair> bps = enumerate_blocks(plan->nv, n_a, n_b);
    const int old_path = plan->path;
    plan->path = 0;
    if (layout_for(*plan, max_pairs_of(bps)).total > plan->budget) {
        plan->path = old_path;
        return LADDER_ERR_BUDGET;
    }
    const int rc = apply_blocking(*plan, n_a, n_b);
    if (rc != LADDER_OK) plan->path = old_path;
    return rc;
}

int ladder_shard_blocks(int n_blocks, const long long* npairs, int world, int* owner) {
    if (n_blocks < 0 || world < 1 || (n_blocks > 0 && (!npairs || !owner))) return LADDER_ERR_ARG;
    const std::vector<int> o = shard_owner(std::vector<long long>(npairs, npairs + n_blocks), world);
    for (int i = 0; i < n_blocks; ++i) owner[i] = o[i];
    return LADDER_OK;
}

int ladder_plan_shard(ladder_plan_t plan, int rank, int world) {
    if (!plan || plan->batched || world < 1 || rank < 0 || rank >= world) return LADDER_ERR_ARG;
    if (plan->shard_world > 1) return LADDER_ERR_ARG;  // already a shard
    if (world == 1) return LADDER_OK;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return LADDER_ERR_CUDA;
    if (plan->path == 1) {   // sharding splits block pairs of the rebuild order
        plan->path = 0;
        if (plan->bps.empty() && choose_blocking(*plan) != LADDER_OK) {
            plan->path = 1;
            return LADDER_ERR_BUDGET;
        }
    }
    int na = 0, nb = 0;
    std::vector<BlockPair> mine;
    const int rc = shard_select(*plan, rank, world, &na, &nb, &mine);
    if (rc != LADDER_OK) return rc;
    plan->n_a = na;
    plan->n_b = nb;
    plan->bps = std::move(mine);
    plan->max_pairs = (int)max_pairs_of(plan->bps);
    plan->ws = layout_for(*plan, plan->max_pairs);
    plan->shard_rank = rank;
    plan->shard_world = world;
    return build_tables(*plan);
}

int ladder_plan_set_form(ladder_plan_t plan, int form) {
    if (!plan || plan->batched || (form != 0 && form != 1)) return LADDER_ERR_ARG;
    if (form == 0 && plan->pb > 0 && plan->pb < plan->nchol) return LADDER_ERR_ARG;   // batches need form 1
    if (form == 1 && plan->precision == LADDER_FP64) return LADDER_ERR_UNSUPPORTED;
    if (form == plan->form) return LADDER_OK;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return LADDER_ERR_CUDA;
    const int old = plan->form;
    plan->form = form;
    // keep the blocking when it still fits, else choose again under the same budget
    int rc = apply_blocking(*plan, plan->n_a, plan->n_b);
    if (rc == LADDER_ERR_BUDGET) rc = choose_blocking(*plan);
    if (rc != LADDER_OK) {
        plan->form = old;
        apply_blocking(*plan, plan->n_a, plan->n_b);
    }
    return rc;
}

int ladder_plan_get_form(ladder_plan_t plan) { return plan ? plan->form : -1; }

int ladder_form_model(int no, int nv, int nchol, int nslices) {
    if (no < 1 || nv < 1 || nchol < 1) return -1;
    if (nslices == 0) nslices = ladder::kDefaultSlices;
    if (nslices < 5 || nslices > 8) return -1;
    return auto_form(no, nv, nchol, nslices);
}

int ladder_plan_set_path(ladder_plan_t plan, int path) {
    if (!plan || plan->batched || path < 0 || path > 2) return LADDER_ERR_ARG;
    if (path != 0 && plan->precision != LADDER_FP64) return LADDER_ERR_UNSUPPORTED;
    if (path == plan->path) return LADDER_OK;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return LADDER_ERR_CUDA;
    if (path == 1) {
        if (plan->shard_world > 1) return LADDER_ERR_ARG;   // a shard holds block pairs only
        return use_factorised(*plan);
    }
    if (path == 2) return use_fused(*plan);
    const int old_path = plan->path;
    plan->path = 0;
    int rc = plan->bps.empty() ? LADDER_ERR_BUDGET : LADDER_OK;
    if (rc == LADDER_OK) {
        const ladder::WsLayout w = layout_for(*plan, plan->max_pairs);
        if (w.total <= plan->budget) plan->ws = w; else rc = LADDER_ERR_BUDGET;
    }
    if (rc == LADDER_ERR_BUDGET) rc = choose_blocking(*plan);
    if (rc != LADDER_OK) {
        plan->path = old_path;
        plan->ws = layout_for(*plan, old_path == 1 ? 0 : plan->max_pairs);
    }
    return rc;
}

int ladder_plan_get_path(ladder_plan_t plan) { return plan ? plan->path : -1; }

int ladder_path_model(int no, int nv, int nchol, int precision) {
    if (no < 1 || nv < 1 || nchol < 1) return -1;
    if (precision != LADDER_FP64 && precision != LADDER_EMU_BF16) return -1;
    return auto_path(no, nv, nchol, precision);
}

size_t ladder_workspace_bytes(ladder_plan_t plan) {
    if (!plan) return 0;
    return plan->ws.total;
}

int ladder_plan_describe(ladder_plan_t plan, int* n_a, int* n_b, int* n_block_pairs, int* max_pairs_per_block,
                         int* nslices, int* precision) {
    if (!plan) return LADDER_ERR_ARG;
    if (n_a) *n_a = plan->n_a;
    if (n_b) *n_b = plan->n_b;
    if (n_block_pairs) *n_block_pairs = (int)plan->bps.size();
    if (max_pairs_per_block) *max_pairs_per_block = plan->max_pairs;
    if (nslices) *nslices = plan->nslices;
    if (precision) *precision = plan->precision;
    return LADDER_OK;
}

int ladder_apply(ladder_plan_t plan, const double* L, const double* t2, double* R, void* ws,
                 cudaStream_t stream) {
    if (!plan || plan->batched || !L || !t2 || !R || !ws) return LADDER_ERR_ARG;
    if (!aligned256(L) || !aligned256(t2) || !aligned256(R) || !aligned256(ws)) return LADDER_ERR_ARG;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return LADDER_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    if (plan->path == 1) {
        e = ladder::launch_fp64_factorised(*plan, L, t2, R, ws, stream);
    } else if (plan->path == 2) {
        for (const auto& bp : plan->bps) {
            e = ladder::launch_fp64_fused(*plan, bp, L, t2, R, stream);
            if (e != cudaSuccess) break;
        }
    } else if (plan->precision == LADDER_FP64) {
        for (const auto& bp : plan->bps) {
            e = ladder::launch_fp64_block(*plan, bp, L, t2, R, ws, stream);
            if (e != cudaSuccess) break;
        }
    } else {
        e = ladder::launch_emu_prep(*plan, L, t2, ws, stream);
        if (e == cudaSuccess) {
            for (const auto& bp : plan->bps) {
                e = ladder::launch_emu_block(*plan, bp, L, R, ws, stream);
                if (e != cudaSuccess) break;
            }
        }
    }
    return map_cuda(e);
}

// Staging of ladder_apply_host: two sets, each L [nchol][nv][nv], t2 and R [no][no][nv][nv].
struct StageLayout {
    size_t t = 0, R = 0, set = 0;   // offsets of t2 and R in a set, bytes per set (L at 0)
};
static StageLayout stage_layout(const ladder_plan_s& p) {
    using ladder::align_up;
    using ladder::kAlign;
    const size_t nv2 = (size_t)p.nv * p.nv;
    StageLayout s;
    s.t = align_up(sizeof(double) * (size_t)p.nchol * nv2, kAlign);
    s.R = s.t + align_up(sizeof(double) * (size_t)p.no * p.no * nv2, kAlign);
    s.set = s.R + align_up(sizeof(double) * (size_t)p.no * p.no * nv2, kAlign);
    return s;
}

size_t ladder_host_staging_bytes(ladder_plan_t plan) {
    if (!plan || plan->batched) return 0;
    return 2 * stage_layout(*plan).set;
}

int ladder_apply_host(ladder_plan_t plan, const double* L_host, const double* t2_host, double* R_host,
                      void* stage, void* ws, cudaStream_t stream) {
    if (!plan || plan->batched || !L_host || !t2_host || !R_host || !stage || !ws) return LADDER_ERR_ARG;
    if (!aligned256(stage) || !aligned256(ws)) return LADDER_ERR_ARG;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return LADDER_ERR_CUDA;
    if (!plan->h2d_stream) {   // first call: the copy stream and its events, all or nothing
        cudaStream_t hs = nullptr;
        cudaEvent_t ev[4] = {};
        bool ok = cudaStreamCreateWithFlags(&hs, cudaStreamNonBlocking) == cudaSuccess;
        for (int i = 0; i < 4 && ok; ++i) ok = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            for (auto e : ev)
                if (e) cudaEventDestroy(e);
            if (hs) cudaStreamDestroy(hs);
            return LADDER_ERR_CUDA;
        }
        plan->host_ready[0] = ev[0];
        plan->host_ready[1] = ev[1];
        plan->host_free[0] = ev[2];
        plan->host_free[1] = ev[3];
        plan->h2d_stream = hs;
    }
    const StageLayout sl = stage_layout(*plan);
    const int s = plan->host_parity;
    char* set = static_cast<char*>(stage) + (size_t)s * sl.set;
    double* Ld = reinterpret_cast<double*>(set);
    double* td = reinterpret_cast<double*>(set + sl.t);
    double* Rd = reinterpret_cast<double*>(set + sl.R);
    const size_t nv2 = (size_t)plan->nv * plan->nv;
    const size_t bL = sizeof(double) * (size_t)plan->nchol * nv2, bT = sizeof(double) * (size_t)plan->no * plan->no * nv2;
    // Inputs into set s on the copy stream, once the call two back (the last one to use set s)
    // has finished with them: so these copies overlap the previous call's contraction.
    cudaStream_t h = plan->h2d_stream;
    if (cudaStreamWaitEvent(h, plan->host_free[s], 0) != cudaSuccess ||
        cudaMemcpyAsync(Ld, L_host, bL, cudaMemcpyHostToDevice, h) != cudaSuccess ||
        cudaMemcpyAsync(td, t2_host, bT, cudaMemcpyHostToDevice, h) != cudaSuccess ||
        cudaEventRecord(plan->host_ready[s], h) != cudaSuccess ||
        cudaStreamWaitEvent(stream, plan->host_ready[s], 0) != cudaSuccess ||
        cudaMemsetAsync(Rd, 0, bT, stream) != cudaSuccess)
        return LADDER_ERR_CUDA;
    const int rc = ladder_apply(plan, Ld, td, Rd, ws, stream);
    if (rc != LADDER_OK) return rc;
    if (cudaEventRecord(plan->host_free[s], stream) != cudaSuccess ||
        cudaMemcpyAsync(R_host, Rd, bT, cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return LADDER_ERR_CUDA;
    plan->host_parity = s ^ 1;
    return LADDER_OK;
}

int ladder_energy(ladder_plan_t plan, const double* t2, const double* R, double* E_dev, double* E_host,
                  cudaStream_t stream) {
    if (!plan || plan->batched || !t2 || !R || (!E_dev && !E_host)) return LADDER_ERR_ARG;
    if (!aligned256(t2) || !aligned256(R)) return LADDER_ERR_ARG;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return LADDER_ERR_CUDA;
    double* target = E_dev ? E_dev : plan->d_partials + plan->n_partials;
    cudaError_t e = ladder::launch_energy(*plan, t2, R, target, stream);
    if (e != cudaSuccess) return LADDER_ERR_CUDA;
    if (E_host) {
        e = cudaMemcpyAsync(E_host, target, sizeof(double), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return LADDER_ERR_CUDA;
    }
    return LADDER_OK;
}

int ladder_plan_batched(ladder_plan_t* out, int n, const int* no, const int* nv, const int* nchol, int precision,
                        int nslices, size_t ws_budget_bytes, int device) {
    if (!out) return LADDER_ERR_ARG;
    *out = nullptr;
    if (n < 1 || !no || !nv || !nchol) return LADDER_ERR_ARG;
    auto* p = new (std::nothrow) ladder_plan_s();
    if (!p) return LADDER_ERR_CUDA;
    p->batched = true;
    p->precision = precision;
    p->device = device;
    size_t budget = ws_budget_bytes;
    if (budget == 0) {
        DeviceGuard g0(device);
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            destroy_plan(p);
            return LADDER_ERR_CUDA;
        }
        budget = (size_t)((double)free_b * 0.98 * 0.9);
    }
    // Every instance is planned against the whole budget (one block pair whenever its packed
    // ERI fits), and the plan's workspace holds as many instances at once as the budget allows.
    for (int k = 0; k < n; ++k) {
        ladder_plan_s* s = nullptr;
        const int rc = make_plan(&s, no[k], nv[k], nchol[k], precision, nslices, budget, device, true, false);
        if (rc != LADDER_OK) {
            destroy_plan(p);
            return rc;
        }
        p->sub.push_back(s);
        p->model_s.push_back(plan_time(*s));
    }
    p->nslices = p->sub[0]->nslices;
    p->num_sms = p->sub[0]->num_sms;
    p->budget = budget;
    size_t biggest = ladder::kAlign, sum = 0;
    for (auto* s : p->sub) {
        biggest = std::max(biggest, ladder::align_up(s->ws.total, ladder::kAlign));
        sum += ladder::align_up(s->ws.total, ladder::kAlign);
    }
    p->ws.total = std::max(biggest, std::min(sum, ladder::align_up(budget, ladder::kAlign)));
    const int max_streams = (int)std::max<size_t>(1, std::min<size_t>(std::min(n, 8), p->ws.total / biggest));
    p->max_streams = max_streams;
    DeviceGuard guard(device);
    p->ws_off.resize(max_streams);
    for (int w = 0; w < max_streams; ++w) p->ws_off[w] = (size_t)w * biggest;
    p->workers.resize(max_streams, nullptr);
    p->fork_join.resize(1 + max_streams, nullptr);
    bool ok = true;
    for (auto& w : p->workers) ok = ok && cudaStreamCreateWithFlags(&w, cudaStreamNonBlocking) == cudaSuccess;
    for (auto& e : p->fork_join) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaMalloc(&p->d_status, sizeof(unsigned)) == cudaSuccess &&
         cudaMemset(p->d_status, 0, sizeof(unsigned)) == cudaSuccess;
    if (!ok) {
        destroy_plan(p);
        return LADDER_ERR_CUDA;
    }
    int rc = LADDER_OK;
    if (precision != LADDER_FP64) {
        // Default: the instances in as few groups as the workspace allows.
        rc = schedule_groups(*p, p->ws.total);
    } else {
        // Default from the model: enough streams that the largest instance is the tail.
        double total = 0.0, largest = 0.0;
        for (double t : p->model_s) {
            total += t;
            largest = std::max(largest, t);
        }
        schedule_batched(*p, (int)std::ceil(total / std::max(largest, 1e-12)));
    }
    if (rc != LADDER_OK) {
        destroy_plan(p);
        return rc;
    }
    *out = p;
    return LADDER_OK;
}

int ladder_batched_schedule(ladder_plan_t plan, int schedule, int* groups_or_streams) {
    if (!plan || !plan->batched || schedule == 0) return LADDER_ERR_ARG;
    if (schedule < 0 && plan->precision == LADDER_FP64) return LADDER_ERR_ARG;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return LADDER_ERR_CUDA;
    if (schedule > 0) {
        schedule_batched(*plan, std::min(schedule, plan->max_streams));
    } else {
        const int rc = schedule_groups(*plan, plan->ws.total / (size_t)(-(long long)schedule));
        if (rc != LADDER_OK) return rc;
    }
    if (groups_or_streams) *groups_or_streams = plan->sched_groups > 0 ? -plan->sched_groups : plan->nstreams;
    return LADDER_OK;
}

int ladder_apply_batched(ladder_plan_t plan, const double* const* L, const double* const* t2, double* const* R,
                         void* ws, cudaStream_t stream) {
    if (!plan || !plan->batched || !L || !t2 || !R || !ws) return LADDER_ERR_ARG;
    if (!aligned256(ws)) return LADDER_ERR_ARG;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return LADDER_ERR_CUDA;
    if (plan->sched_groups > 0) {
        // Grouped schedule: each group is one ERI launch and one ladder launch per shape.
        char* base = static_cast<char*>(ws);
        for (size_t g = 0; g < plan->groups.size(); ++g) {
            const std::vector<int>& grp = plan->groups[g];
            if (grp.size() == 1 && !groupable(*plan->sub[grp[0]])) {
                const int k = grp[0];
                const int rc = ladder_apply(plan->sub[k], L[k], t2[k], R[k], base + plan->inst_off[k], stream);
                if (rc != LADDER_OK) return rc;
                continue;
            }
            std::vector<const ladder_plan_s*> subs;
            std::vector<void*> wsv;
            std::vector<const double*> Lv, tv;
            std::vector<double*> Rv;
            for (int k : grp) {
                if (!L[k] || !t2[k] || !R[k] || !aligned256(L[k]) || !aligned256(t2[k]) || !aligned256(R[k]))
                    return LADDER_ERR_ARG;
                subs.push_back(plan->sub[k]);
                wsv.push_back(base + plan->inst_off[k]);
                Lv.push_back(L[k]);
                tv.push_back(t2[k]);
                Rv.push_back(R[k]);
            }
            const int4* entries = static_cast<const int4*>(plan->d_group_entries) + plan->group_eoff[g];
            const cudaError_t e = ladder::launch_emu_group(*plan, subs.data(), (int)subs.size(), wsv.data(),
                                                           Lv.data(), tv.data(), Rv.data(), entries,
                                                           plan->group_ecnt[g], stream);
            if (e != cudaSuccess) return LADDER_ERR_CUDA;
        }
        return LADDER_OK;
    }
    const int k = plan->nstreams;
    // fork: every worker stream waits for the work already queued on the caller's stream
    if (cudaEventRecord(plan->fork_join[0], stream) != cudaSuccess) return LADDER_ERR_CUDA;
    for (int w = 0; w < k; ++w)
        if (cudaStreamWaitEvent(plan->workers[w], plan->fork_join[0], 0) != cudaSuccess) return LADDER_ERR_CUDA;
    int rc = LADDER_OK;
    for (int i : plan->order) {
        const int w = plan->stream_of[i];
        rc = ladder_apply(plan->sub[i], L[i], t2[i], R[i], static_cast<char*>(ws) + plan->ws_off[w],
                          plan->workers[w]);
        if (rc != LADDER_OK) break;
    }
    // join: the caller's stream waits for every worker
    for (int w = 0; w < k; ++w) {
        if (cudaEventRecord(plan->fork_join[1 + w], plan->workers[w]) != cudaSuccess ||
            cudaStreamWaitEvent(stream, plan->fork_join[1 + w], 0) != cudaSuccess)
            return LADDER_ERR_CUDA;
    }
    return rc;
}

int ladder_tune_batched(ladder_plan_t plan, const double* const* L, const double* const* t2, double* const* R,
                        void* ws, cudaStream_t stream, int* best_schedule) {
    if (!plan || !plan->batched) return LADDER_ERR_ARG;
    DeviceGuard guard(plan->device);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LADDER_ERR_CUDA;
    // Candidates: worker-stream schedules with 1, 2, 4, ... streams, and (emulated path) grouped
    // schedules with the whole workspace, a half and a quarter of it per group.
    struct Cand { int streams; size_t cap; int bn = ladder::kEmuTileN; };
    std::vector<Cand> cands;
    for (int k = 1; k < plan->max_streams; k *= 2) cands.push_back({k, 0});
    cands.push_back({plan->max_streams, 0});
    if (plan->precision != LADDER_FP64) {
        size_t biggest = 0;
        for (auto* s : plan->sub) biggest = std::max(biggest, ladder::align_up(s->ws.total, ladder::kAlign));
        for (int d = 1; d <= 4; d *= 2)
            if (plan->ws.total / d >= biggest) cands.push_back({0, plan->ws.total / d});
    }
    // Ladder column tile on one SM: 96 pairs (the widest that the five accumulators leave room
    // for in TMEM) or 64 (more, smaller tiles for instances with few pairs).
    const int widths[2] = {ladder::kEmuTileN, 64};
    const int nwidths = plan->precision != LADDER_FP64 ? 2 : 1;
    {
        const std::vector<Cand> base = cands;
        cands.clear();
        for (int wi = 0; wi < nwidths; ++wi)
            for (Cand c : base) {
                c.bn = widths[wi];
                cands.push_back(c);
            }
    }
    float best_ms = 1e30f;
    Cand best = cands[0];
    int rc = LADDER_OK;
    auto use = [&](const Cand& c) -> int {
        ladder_plan_set_ladder_tile(plan, c.bn);
        if (c.streams > 0) {
            schedule_batched(*plan, c.streams);
            return LADDER_OK;
        }
        return schedule_groups(*plan, c.cap);
    };
    for (const Cand& c : cands) {
        if (rc != LADDER_OK) break;
        if ((rc = use(c)) != LADDER_OK) break;
        rc = ladder_apply_batched(plan, L, t2, R, ws, stream);  // warm-up of this schedule
        if (rc != LADDER_OK) break;
        if (cudaEventRecord(e0, stream) != cudaSuccess) rc = LADDER_ERR_CUDA;
        if (rc == LADDER_OK) rc = ladder_apply_batched(plan, L, t2, R, ws, stream);
        if (rc == LADDER_OK && (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
            rc = LADDER_ERR_CUDA;
        float ms = 0.0f;
        if (rc == LADDER_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = LADDER_ERR_CUDA;
        // A grouped schedule (fewer launches) wins ties within 1 %.
        const float score = c.streams > 0 ? ms : ms * 0.99f;
        if (rc == LADDER_OK && score < best_ms) {
            best_ms = score;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int rc2 = use(best);
    if (rc == LADDER_OK) rc = rc2;
    if (best_schedule) *best_schedule = plan->sched_groups > 0 ? -plan->sched_groups : plan->nstreams;
    return rc;
}

int ladder_plan_set_pbatch(ladder_plan_t plan, int pb) {
    if (!plan || plan->batched || plan->shard_world > 1 || pb < 0 || pb % 64 != 0) return LADDER_ERR_ARG;
    if (plan->precision == LADDER_FP64) return pb == 0 ? LADDER_OK : LADDER_ERR_UNSUPPORTED;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return LADDER_ERR_CUDA;
    const int old_pb = plan->pb, old_form = plan->form;
    plan->pb = pb >= plan->nchol ? 0 : pb;
    if (plan->pb > 0) plan->form = 1;   // batches add into the split form's int64 V
    int rc = apply_blocking(*plan, plan->n_a, plan->n_b);
    if (rc == LADDER_ERR_BUDGET) rc = choose_blocking(*plan);
    if (rc != LADDER_OK) {
        plan->pb = old_pb;
        plan->form = old_form;
        apply_blocking(*plan, plan->n_a, plan->n_b);
    }
    return rc;
}

int ladder_plan_get_pbatch(ladder_plan_t plan) { return plan ? (plan->pb > 0 && plan->pb < plan->nchol ? plan->pb : 0) : -1; }

int ladder_plan_set_eri_chunk(ladder_plan_t plan, int blocks) {
    if (!plan || blocks < 1 || blocks > 4) return LADDER_ERR_ARG;
    plan->eri_chunk_max = blocks;
    for (auto* s : plan->sub) s->eri_chunk_max = blocks;
    return LADDER_OK;
}

int ladder_plan_eri_chunk(ladder_plan_t plan, const void* ws, cudaStream_t stream) {
    if (!plan || plan->batched || !ws || plan->precision == LADDER_FP64 || plan->path != 0) return -1;
    DeviceGuard guard(plan->device);
    int kbc = 0;
    if (cudaMemcpyAsync(&kbc, static_cast<const char*>(ws) + plan->ws.eri_kbc, sizeof(int), cudaMemcpyDeviceToHost,
                        stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return -1;
    return kbc * ladder::emu_eri_stage_k(plan->nslices);
}

int ladder_plan_set_ladder_tile(ladder_plan_t plan, int bn) {
    if (!plan || bn < 16 || bn > ladder::kEmuTileN || bn % 16 != 0) return LADDER_ERR_ARG;
    plan->lad_bn = bn;
    for (auto* s : plan->sub) s->lad_bn = bn;
    return LADDER_OK;
}

int ladder_plan_get_ladder_tile(ladder_plan_t plan) { return plan ? plan->lad_bn : -1; }

int ladder_plan_set_wait_limit(ladder_plan_t plan, double seconds) {
    if (!plan || !(seconds >= 0.0) || seconds > 3600.0) return LADDER_ERR_ARG;
    if (seconds > 0.0 && seconds < 1e-3) return LADDER_ERR_ARG;
    const unsigned long long ns =
        seconds == 0.0 ? ladder::kDefaultWaitNs : (unsigned long long)std::llround(seconds * 1e9);
    plan->wait_ns = ns;
    for (auto* s : plan->sub) s->wait_ns = ns;
    return LADDER_OK;
}

double ladder_plan_get_wait_limit(ladder_plan_t plan) { return plan ? (double)plan->wait_ns * 1e-9 : -1.0; }

int ladder_plan_set_timing(ladder_plan_t plan, int enable) {
    if (!plan) return LADDER_ERR_ARG;
    DeviceGuard guard(plan->device);
    std::vector<ladder_plan_s*> all{plan};
    for (auto* s : plan->sub) all.push_back(s);
    for (auto* q : all) {
        free_events(q);
        if (!enable) continue;
        const size_t slots = 64 * (q->bps.size() + 8);
        q->ev_pool.resize(2 * slots);
        q->ev_kind.assign(slots, -1);
        q->ev_kernels.assign(slots, 0);
        for (auto& e : q->ev_pool)
            if (cudaEventCreate(&e) != cudaSuccess) {
                free_events(q);
                return LADDER_ERR_CUDA;
            }
        q->timing = true;
    }
    return LADDER_OK;
}

int ladder_plan_timing(ladder_plan_t plan, int kernel_class, float* total_ms, int* launches, int reset) {
    if (!plan || kernel_class < 0 || kernel_class >= LADDER_KERNEL_CLASSES) return LADDER_ERR_ARG;
    DeviceGuard guard(plan->device);
    std::vector<ladder_plan_s*> all{plan};
    for (auto* s : plan->sub) all.push_back(s);
    float sum = 0.0f;
    int n = 0;
    for (auto* q : all) {
        for (size_t k = 0; k < q->ev_used; ++k) {
            if (q->ev_kind[k] != kernel_class) continue;
            if (cudaEventSynchronize(q->ev_pool[2 * k + 1]) != cudaSuccess) return LADDER_ERR_CUDA;
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, q->ev_pool[2 * k], q->ev_pool[2 * k + 1]) != cudaSuccess)
                return LADDER_ERR_CUDA;
            sum += ms;
            n += q->ev_kernels[k];
        }
        if (reset) q->ev_used = 0;
    }
    if (total_ms) *total_ms = sum;
    if (launches) *launches = n;
    return LADDER_OK;
}

int ladder_last_status(ladder_plan_t plan, cudaStream_t stream) {
    if (!plan) return LADDER_ERR_ARG;
    DeviceGuard guard(plan->device);
    unsigned word = 0;
    std::vector<ladder_plan_s*> all{plan};
    for (auto* s : plan->sub) all.push_back(s);
    for (auto* q : all) {
        if (!q->d_status) continue;
        unsigned w = 0;
        if (cudaMemcpyAsync(&w, q->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess ||
            cudaMemsetAsync(q->d_status, 0, sizeof(unsigned), stream) != cudaSuccess)
            return LADDER_ERR_CUDA;
        word |= w;
    }
    if (word & ladder::kStatusBounds) return LADDER_ERR_BOUNDS;
    if (word & ladder::kStatusTimeout) return LADDER_ERR_TIMEOUT;
    if (word & ladder::kStatusNumeric) return LADDER_ERR_NUMERIC;
    return LADDER_OK;
}

void ladder_plan_destroy(ladder_plan_t plan) { destroy_plan(plan); }

}  // extern "C"

namespace {

// Host-only plan of ladder_plan_dry / ladder_plan_shard_dry: the blocking ladder_plan would
// choose (or the forced one), with no CUDA call.
int dry_plan(ladder_plan_s& p, int no, int nv, int nchol, int precision, int nslices, size_t ws_budget_bytes,
             int num_sms, int force_n_a, int force_n_b) {
    if (no < 1 || nv < 1 || nchol < 1 || num_sms < 1 || ws_budget_bytes == 0) return LADDER_ERR_ARG;
    if (precision == LADDER_EMU_INT8) return LADDER_ERR_UNSUPPORTED;
    if (precision != LADDER_FP64 && precision != LADDER_EMU_BF16) return LADDER_ERR_ARG;
    if (nslices == 0) nslices = ladder::kDefaultSlices;
    if (precision == LADDER_EMU_BF16 && (nslices < 5 || nslices > 8)) return LADDER_ERR_ARG;
    p.no = no;
    p.nv = nv;
    p.nchol = nchol;
    p.precision = precision;
    p.nslices = precision == LADDER_FP64 ? 0 : nslices;
    p.num_sms = num_sms;
    p.budget = ws_budget_bytes;
    p.form = precision == LADDER_FP64 ? 0 : auto_form(no, nv, nchol, nslices);
    int na = force_n_a, nb = force_n_b;
    if (na <= 0 || nb <= 0) {
        int rc = select_blocking(p, &na, &nb);
        if (rc == LADDER_ERR_BUDGET && p.form == 1) {
            p.form = 0;
            rc = select_blocking(p, &na, &nb);
        }
        if (rc == LADDER_OK || rc == LADDER_ERR_BUDGET) {   // batches of Cholesky vectors, as ladder_plan
            if (rc == LADDER_OK) p.bps = enumerate_blocks(nv, na, nb);
            int bna = 0, bnb = 0;
            const int pb = select_pbatch(p, rc == LADDER_OK, &bna, &bnb);
            if (pb > 0) {
                p.pb = pb;
                p.form = 1;
                na = bna;
                nb = bnb;
                rc = LADDER_OK;
            }
        }
        if (rc != LADDER_OK) return rc;
    } else if (na > nv || nb > nv) {
        return LADDER_ERR_ARG;
    }
    p.bps = enumerate_blocks(nv, na, nb);
    p.n_a = na;
    p.n_b = nb;
    if (layout_for(p, max_pairs_of(p.bps)).total > p.budget) return LADDER_ERR_BUDGET;
    return LADDER_OK;
}

void dry_outputs(const ladder_plan_s& p, const std::vector<BlockPair>& bps, int* n_a, int* n_b, size_t* ws_bytes,
                 int max_blocks, int* n_block_pairs, int* blocks) {
    if (n_a) *n_a = p.n_a;
    if (n_b) *n_b = p.n_b;
    if (ws_bytes) *ws_bytes = layout_for(p, max_pairs_of(bps)).total;
    if (n_block_pairs) *n_block_pairs = (int)bps.size();
    if (blocks) {
        for (int k = 0; k < (int)bps.size() && k < max_blocks; ++k) {
            blocks[5 * k + 0] = bps[k].a0;
            blocks[5 * k + 1] = bps[k].a1;
            blocks[5 * k + 2] = bps[k].b0;
            blocks[5 * k + 3] = bps[k].b1;
            blocks[5 * k + 4] = bps[k].npairs;
        }
    }
}

}  // namespace

extern "C" {

int ladder_plan_dry(int no, int nv, int nchol, int precision, int nslices, size_t ws_budget_bytes, int num_sms,
                    int force_n_a, int force_n_b, int* n_a, int* n_b, size_t* ws_bytes, int max_blocks,
                    int* n_block_pairs, int* blocks) {
    ladder_plan_s p;
    const int rc = dry_plan(p, no, nv, nchol, precision, nslices, ws_budget_bytes, num_sms, force_n_a, force_n_b);
    if (rc != LADDER_OK) return rc;
    dry_outputs(p, p.bps, n_a, n_b, ws_bytes, max_blocks, n_block_pairs, blocks);
    return LADDER_OK;
}

int ladder_plan_shard_dry(int no, int nv, int nchol, int precision, int nslices, size_t ws_budget_bytes,
                          int num_sms, int rank, int world, int* n_a, int* n_b, size_t* ws_bytes, int max_blocks,
                          int* n_block_pairs, int* blocks) {
    if (world < 1 || rank < 0 || rank >= world) return LADDER_ERR_ARG;
    ladder_plan_s p;
    int rc = dry_plan(p, no, nv, nchol, precision, nslices, ws_budget_bytes, num_sms, 0, 0);
    if (rc != LADDER_OK) return rc;
    if (world > 1) {
        int na = 0, nb = 0;
        std::vector<BlockPair> mine;
        if ((rc = shard_select(p, rank, world, &na, &nb, &mine)) != LADDER_OK) return rc;
        p.n_a = na;
        p.n_b = nb;
        p.bps = std::move(mine);
    }
    dry_outputs(p, p.bps, n_a, n_b, ws_bytes, max_blocks, n_block_pairs, blocks);
    return LADDER_OK;
}

const char* ladder_strerror(int status) {
    switch (status) {
        case LADDER_OK: return "ok";
        case LADDER_ERR_ARG: return "invalid argument (size, alignment or null pointer)";
        case LADDER_ERR_BUDGET: return "no a/b blocking fits the workspace budget";
        case LADDER_ERR_CUDA: return "CUDA runtime error";
        case LADDER_ERR_UNSUPPORTED: return "unsupported configuration";
        case LADDER_ERR_TIMEOUT: return "a kernel's bounded wait timed out";
        case LADDER_ERR_NUMERIC: return "a kernel consistency check failed";
        case LADDER_ERR_BOUNDS: return "an index check of a LADDER_CHECK build failed";
        default: return "unknown status";
    }
}

double ladder_flops(int no, int nv, int nchol) {
    const double p = 0.5 * (double)nv * (nv + 1);
    const double nv2 = (double)nv * nv;
    return 2.0 * nchol * nv2 * p + 2.0 * (double)no * no * nv2 * p;
}

}  // extern "C"
