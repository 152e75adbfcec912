// Plan construction (host orchestration) and the C ABI entry points.
//
// A plan holds, on the device: Morton-sorted points and weights, the octree
// (leaves, neighbour lists, interaction lists grouped by translation offset), all
// translation operators, and the sparse self/near correction.  The octree is uniform
// (every leaf at the smallest depth that holds leaf_max points) or, with the adaptive
// option, split box by box with U / V / W / X lists for leaves of unequal depth.
// The sort, the per-point leaf data, the neighbour and interaction lists of a uniform
// tree, the operators and the correction are built by device kernels; the host keeps
// the per-level box tables, builds the adaptive lists, and turns lists into work items.
// Sec. 2.2 (discretisation, singular treatment), Sec. 2.3 (octree, sweeps),
// Sec. 3.1-3.2 (Morton order, cell = index + count).
#include <algorithm>
#include <functional>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>
#include <string>
#include <vector>

#include "hfmm_internal.cuh"
#include "kernel_poly.h"

using namespace hfmm;

static thread_local std::string g_last_error;

void hfmm_set_last_error(const std::string& msg) { g_last_error = msg; }

static inline uint64_t spread3_h(uint64_t v) {
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffull;
    v = (v | v << 16) & 0x1f0000ff0000ffull;
    v = (v | v << 8) & 0x100f00f00f00f00full;
    v = (v | v << 4) & 0x10c30c30c30c30c3ull;
    v = (v | v << 2) & 0x1249249249249249ull;
    return v;
}
static inline uint64_t morton_h(uint64_t x, uint64_t y, uint64_t z) {
    return (spread3_h(x) << 2) | (spread3_h(y) << 1) | spread3_h(z);
}
static inline uint64_t compact3_h(uint64_t v) {
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffff;
    return v;
}
static inline void demorton_h(uint64_t k, int64_t* c) {
    c[0] = (int64_t)compact3_h(k >> 2);
    c[1] = (int64_t)compact3_h(k >> 1);
    c[2] = (int64_t)compact3_h(k);
}

static int64_t find_sorted(const std::vector<uint64_t>& keys, uint64_t key) {
    auto it = std::lower_bound(keys.begin(), keys.end(), key);
    if (it == keys.end() || *it != key) return -1;
    return (int64_t)(it - keys.begin());
}

// projection radius in [0.55 a, a] keeping every j_n(k rho), n <= p, away from a zero
static double choose_rho(double k, double a, int p) {
    std::vector<double> re(p + 1), im(p + 1);
    double best = a, best_score = -1.0;
    for (int t = 0; t <= 32; ++t) {
        double rho = a * (1.0 - 0.45 * t / 32.0);
        host_hn_scaled(p, k * rho, 1.0, re.data(), im.data());
        double sc = 1e300;
        for (int n = 0; n <= p; ++n) sc = std::min(sc, std::fabs(re[n]) / std::hypot(re[n], im[n]));
        if (sc > best_score * 1.0000001) {
            best_score = sc;
            best = rho;
        }
    }
    return best;
}

static int level_order(const hfmm_config& c, double k, double side) {
    if (c.p_fixed > 0) return c.p_fixed;
    double ka = k * 0.5 * std::sqrt(3.0) * side;
    int p = (int)std::ceil(ka + 6.0 * std::log10(ka + 3.14159265358979323846));
    return std::max(p, c.p_min);
}

namespace {
struct HostLevel {
    std::vector<uint64_t> key;
    std::vector<int32_t> start;  // uniform: nbox + 1 (boxes cover the points); adaptive: nbox
    std::vector<int32_t> end;    // adaptive: end of each box's point range
    std::vector<int32_t> leaf;   // adaptive: leaf index of each box, -1 for a split box
};

// every occupied cell of level l of the sorted keys (20 bits per axis)
static HostLevel occupied_cells(const std::vector<uint64_t>& skeys, int l) {
    HostLevel h;
    const int sh = 3 * (20 - l);
    for (size_t i = 0; i < skeys.size(); ++i) {
        const uint64_t key = skeys[i] >> sh;
        if (i == 0 || key != (skeys[i - 1] >> sh)) {
            h.key.push_back(key);
            h.start.push_back((int32_t)i);
        }
    }
    h.start.push_back((int32_t)skeys.size());
    return h;
}

// (source, destination) column pairs grouped by operator: bucket g is
// pairs[start[g] .. start[g + 1])
struct PairBuckets {
    std::vector<int2> pairs;
    std::vector<int64_t> start;
    int64_t size(size_t g) const { return start[g + 1] - start[g]; }
    static PairBuckets from(const std::vector<std::vector<int2>>& b) {
        PairBuckets pb;
        pb.start.assign(b.size() + 1, 0);
        for (size_t g = 0; g < b.size(); ++g) {
            pb.pairs.insert(pb.pairs.end(), b[g].begin(), b[g].end());
            pb.start[g + 1] = (int64_t)pb.pairs.size();
        }
        return pb;
    }
};

// Target-stationary M2L work of one level (m2l_ts.cu): tiles of tt (<= kTsTile) consecutive target
// boxes; in each tile the translations grouped by canonical operator (refl[slot].x) into
// chunks of up to kTsChunkCols columns {source box | rc << 24, target slot * kTsRows | rc << 24},
// the reflection code rc's bits being the x, y, z flips that carry the canonical offset onto
// the slot's offset.  The kernel adds a chunk's columns into the tile eight at a time without
// atomics, so no target may repeat within an aligned group of eight columns (a target meets one
// canonical operator through up to eight reflections): the columns are ordered by (occurrence
// of their target, target), which keeps equal targets apart, and where a repeat would still
// fall into one group the group is closed with padding columns.  Padding columns (source box 0,
// the tile's spare row kTsTrash) also fill every chunk to a multiple of eight columns.
void emit_ts_level(const PairBuckets& pb, const std::vector<int4>& refl, int ncanon, int64_t nbox, int Pl,
                   int64_t bxofs, int64_t lofs, int64_t canon_op, int tt, std::vector<TsTile>& tiles,
                   std::vector<TsChunk>& chunks, std::vector<int2>& cols) {
    const int64_t ntile = (nbox + tt - 1) / tt;
    std::vector<int64_t> start((size_t)(ntile * ncanon + 1), 0);
    for (size_t g = 0; g + 1 < pb.start.size(); ++g)
        for (int64_t e = pb.start[g]; e < pb.start[g + 1]; ++e)
            ++start[(size_t)((pb.pairs[e].y / tt) * ncanon + refl[g].x) + 1];
    for (size_t q = 1; q < start.size(); ++q) start[q] += start[q - 1];
    std::vector<int2> tmp((size_t)start.back());
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (size_t g = 0; g + 1 < pb.start.size(); ++g) {
        const int rc = refl[g].y | (refl[g].z << 1) | (refl[g].w << 2);
        for (int64_t e = pb.start[g]; e < pb.start[g + 1]; ++e) {
            const int2 pr = pb.pairs[e];  // (source, target)
            tmp[(size_t)fill[(size_t)((pr.y / tt) * ncanon + refl[g].x)]++] =
                make_int2(pr.x, (pr.y % tt) | (rc << 16));
        }
    }
    const int2 pad = make_int2(0, kTsTrash * kTsRows);
    std::vector<int> occ((size_t)tt);
    std::vector<std::pair<int64_t, int2>> keyed;
    std::vector<int2> cur;
    for (int64_t t = 0; t < ntile; ++t) {
        TsTile tl{};
        tl.dst = lofs + t * tt * (int64_t)Pl;
        tl.bx = bxofs;
        tl.P = Pl;
        tl.ntgt = (int32_t)std::min<int64_t>(tt, nbox - t * tt);
        tl.chunk0 = (int32_t)chunks.size();
        for (int c = 0; c < ncanon; ++c) {
            const int64_t b = start[(size_t)(t * ncanon + c)], e = start[(size_t)(t * ncanon + c) + 1];
            if (b == e) continue;
            std::fill(occ.begin(), occ.end(), 0);
            keyed.clear();
            for (int64_t q = b; q < e; ++q) {
                const int j = tmp[(size_t)q].y & 0xffff, rc = tmp[(size_t)q].y >> 16;
                const int2 col = make_int2(tmp[(size_t)q].x | (rc << 24), j * kTsRows | (rc << 24));
                keyed.push_back({(int64_t)occ[(size_t)j]++ * tt + j, col});
            }
            std::stable_sort(keyed.begin(), keyed.end(),
                             [](const std::pair<int64_t, int2>& x, const std::pair<int64_t, int2>& y) {
                                 return x.first < y.first;
                             });
            bool first = true;
            cur.clear();
            auto flush = [&]() {
                TsChunk ch{};
                while (cur.size() & 7) cur.push_back(pad);
                ch.op = canon_op + (int64_t)c * kTsOpElems;
                ch.col0 = (int32_t)cols.size();
                ch.ncol = (int16_t)cur.size();
                ch.newop = (int16_t)first;
                first = false;
                cols.insert(cols.end(), cur.begin(), cur.end());
                chunks.push_back(ch);
                cur.clear();
            };
            for (const auto& kc : keyed) {
                const int j = kc.second.y & 0xffffff;
                bool rep = false;
                for (size_t q = cur.size() & ~(size_t)7; q < cur.size(); ++q) rep |= (cur[q].y & 0xffffff) == j;
                if (rep)
                    while (cur.size() & 7) cur.push_back(pad);
                if ((int)cur.size() == kTsChunkCols) flush();
                cur.push_back(kc.second);
            }
            if (!cur.empty()) flush();
        }
        tl.nchunk = (int32_t)chunks.size() - tl.chunk0;
        if (tl.nchunk > 0) tiles.push_back(tl);
    }
}

void emit_items(const PairBuckets& pb, const std::vector<int64_t>& op_of_bucket, int64_t src, int64_t dst, int pin,
                int pout, int atomic, std::vector<TransItem>& items, std::vector<int2>& cols,
                int width = HFMM_TRANS_NB) {
    for (size_t g = 0; g + 1 < pb.start.size(); ++g) {
        const int2* v = pb.pairs.data() + pb.start[g];
        const int64_t nv = pb.size(g);
        for (int64_t c0 = 0; c0 < nv; c0 += width) {
            TransItem it{};
            it.op = op_of_bucket[g];
            it.src = src;
            it.dst = dst;
            it.cols = (int32_t)cols.size();
            it.ncol = (int16_t)std::min<int64_t>(width, nv - c0);
            it.pin = (int16_t)pin;
            it.pout = (int16_t)pout;
            it.atomic = (int16_t)atomic;
            for (int q = 0; q < it.ncol; ++q) cols.push_back(v[c0 + q]);
            items.push_back(it);
        }
    }
}
}  // namespace

// candidates of each tunable (the order of hfmm_plan_tuning's tuned_ms) and the defaults
constexpr int kTuneCount[HFMM_NUM_TUNABLES] = {3, 2, 3, 2};
constexpr int kTuneValue[HFMM_NUM_TUNABLES][HFMM_TUNE_CANDIDATES] = {{0, 1, 2}, {0, 1}, {8, 16, 32}, {0, 1}};
constexpr int kTuneDefault[HFMM_NUM_TUNABLES] = {kDefaultP2PKernel, kDefaultM2LKernel, 32, kDefaultOverlap};

// Splits the source-stationary M2L groups (built with at most m2l_tc_max_group() items,
// one operator each) into groups of at most g items; the M2M / L2L groups follow unchanged.
static void apply_tc_group(hfmm_plan* P, int g, cudaStream_t st) {
    std::vector<int4> out;
    for (int64_t q = 0; q < P->tc_m2l_base; ++q) {
        const int4 b = P->host_groups[(size_t)q];
        for (int o = 0; o < b.y; o += g) out.push_back(make_int4(b.x + o, std::min(g, b.y - o), b.z, b.w));
    }
    const int64_t n_m2l = (int64_t)out.size(), shift = n_m2l - P->tc_m2l_base;
    out.insert(out.end(), P->host_groups.begin() + P->tc_m2l_base, P->host_groups.end());
    P->tc_groups.upload(out, nullptr, st);
    HFMM_CUDA(cudaStreamSynchronize(st));  // `out` is freed on return
    P->n_tc_groups = n_m2l;
    for (size_t l = 0; l < P->m2m_tc_base.size(); ++l) {
        const auto& a = P->m2m_tc_base[l];
        P->m2m_tc[l] = a.second > a.first ? std::make_pair(a.first + shift, a.second + shift) : a;
    }
    for (size_t l = 0; l < P->l2l_tc_base.size(); ++l) {
        const auto& a = P->l2l_tc_base[l];
        P->l2l_tc[l] = a.second > a.first ? std::make_pair(a.first + shift, a.second + shift) : a;
    }
    P->tc_group_used = g;
    P->mvg.reset();
}

// *bad = 1 if any entry is not finite (grid-stride)
__global__ void k_flag_nonfinite(const float2* __restrict__ a, int64_t n, int* __restrict__ bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = a[i];
        if (!isfinite(v.x) || !isfinite(v.y)) *bad = 1;
    }
}

__global__ void k_tune_fill(int64_t N, float2* __restrict__ sig) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint32_t h = (uint32_t)i * 2654435761u + 12345u;  // a multiplicative hash: values in [-1, 1)
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    sig[i] = make_float2((float)(h & 0xffff) / 32768.f - 1.f, (float)(h >> 16) / 32768.f - 1.f);
}

// Plan-time tuning (cfg.autotune = 1), the counterpart of the paper's search for its task size
// and leaf size (Sec. 3.2, 6.2): every choice the configuration left open is timed on this
// plan's own tree and operators, one whole matvec per measurement (CUDA events on the plan's
// stream, one warm-up then the mean of three), and the fastest is kept.  Order: near-field
// kernel, M2L kernel, tensor-core group size (source-stationary M2L only), matvec form.
static void tune_plan(hfmm_plan* P, cudaStream_t st) {
    const hfmm_config& cfg = P->cfg;
    k_tune_fill<<<(unsigned)((P->N + 255) / 256), 256, 0, st>>>(P->N, P->sig.p);
    HFMM_CUDA(cudaGetLastError());
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    HFMM_CUDA(cudaEventCreate(&e0));
    struct Ev {
        cudaEvent_t* a;
        cudaEvent_t* b;
        ~Ev() {
            if (*a) cudaEventDestroy(*a);
            if (*b) cudaEventDestroy(*b);
        }
    } guard{&e0, &e1};
    HFMM_CUDA(cudaEventCreate(&e1));
    const int64_t launches0 = P->launches;
    auto time_matvec = [&]() -> float {
        P->mvg.reset();
        run_matvec_sorted(P, 7, st);  // warm-up (and the graph capture of the two-branch form)
        HFMM_CUDA(cudaEventRecord(e0, st));
        for (int r = 0; r < 3; ++r) run_matvec_sorted(P, 7, st);
        HFMM_CUDA(cudaEventRecord(e1, st));
        HFMM_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        HFMM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        return ms / 3.f;
    };
    auto pick = [&](int a, const std::function<void(int)>& set) {
        for (int c = 0; c < kTuneCount[a]; ++c) {
            set(kTuneValue[a][c]);
            P->tune_ms[a][c] = time_matvec();
        }
        int v = 0;
        if (hfmm_tune_choose(a, P->tune_ms[a], kTuneCount[a], &v) != HFMM_OK) v = kTuneDefault[a];
        set(v);
    };
    const bool staged_p2p = P->poly_p2p && P->p2p_cap > 0 && P->p2p_maxnbr <= 64;
    if (cfg.p2p_kernel < 0 && staged_p2p) pick(0, [&](int v) { P->p2p_variant = v; });
    if (cfg.m2l_kernel < 0 && P->n_ts_tiles > 0 && P->n_tc_groups > 0) pick(1, [&](int v) { P->m2l_variant = v; });
    if (cfg.tc_group == 0 && P->m2l_variant == 0 && P->tc_m2l_base > 0) pick(2, [&](int g) { apply_tc_group(P, g, st); });
    if (cfg.overlap < 0 && !P->adaptive) pick(3, [&](int v) { P->mv_mode = v; });
    P->mvg.reset();
    P->launches = launches0;  // tuning launches are not the caller's
}

static void build_plan(hfmm_plan* P, const double* V, int64_t nv, const int32_t* F, int64_t nt, cudaStream_t st) {
    const hfmm_config& cfg = P->cfg;
    const double k = P->k;
    const int64_t N = 3 * nt;
    P->nt = nt;
    P->N = N;
    // ---------------------------------------------------------- points (Sec. 2.2)
    std::vector<double> X(3 * N), W(N);
    std::vector<int32_t> T(N);
    double edge_sum = 0.0;
    for (int64_t n = 0; n < nt; ++n) {
        const double* v[3];
        for (int a = 0; a < 3; ++a) {
            int32_t id = F[3 * n + a];
            if (id < 0 || id >= nv) throw HfmmError{HFMM_E_MESH, "triangle vertex index out of range"};
            v[a] = V + 3 * (int64_t)id;
            for (int d = 0; d < 3; ++d)
                if (!std::isfinite(v[a][d])) throw HfmmError{HFMM_E_MESH, "non-finite vertex coordinate"};
        }
        double e1[3], e2[3];
        for (int d = 0; d < 3; ++d) {
            e1[d] = v[1][d] - v[0][d];
            e2[d] = v[2][d] - v[0][d];
        }
        double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double area = 0.5 * std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        double l2 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
        if (!(area > 1e-14 * l2) || !(area > 0.0)) throw HfmmError{HFMM_E_MESH, "degenerate (zero-area) triangle"};
        for (int a = 0; a < 3; ++a) {
            double e[3];
            for (int d = 0; d < 3; ++d) e[d] = v[(a + 1) % 3][d] - v[a][d];
            edge_sum += std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
            int64_t i = 3 * n + a;
            for (int d = 0; d < 3; ++d)
                X[3 * i + d] = (2.0 / 3.0) * v[a][d] + (1.0 / 6.0) * v[(a + 1) % 3][d] + (1.0 / 6.0) * v[(a + 2) % 3][d];
            W[i] = area / 3.0;
            T[i] = (int32_t)n;
        }
    }
    P->mean_edge = edge_sum / (3.0 * (double)nt);
    P->r_near = cfg.near_factor * P->mean_edge;
    // ---------------------------------------------------------- octree
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = 0; i < N; ++i)
        for (int d = 0; d < 3; ++d) {
            mn[d] = std::min(mn[d], X[3 * i + d]);
            mx[d] = std::max(mx[d], X[3 * i + d]);
        }
    double ext = std::max(mx[0] - mn[0], std::max(mx[1] - mn[1], mx[2] - mn[2]));
    double D = 1.0;
    if (ext > 0.0) {
        while (D < ext) D *= 2.0;
        while (D * 0.5 >= ext) D *= 0.5;
    }
    P->D = D;
    for (int d = 0; d < 3; ++d) P->lo[d] = 0.5 * (mn[d] + mx[d]) - 0.5 * D;
    const int LMAX = 20;
    const double scale20 = std::ldexp(1.0, LMAX) / D;
    size_t* cnt = &P->dev_bytes;
    // Morton keys and their stable sort on the device; the sorted keys come back for
    // the level tables (a few bytes per box), the permutation stays on the device
    P->x64.upload(X, cnt, st);
    DBuf<uint64_t> d_keys;
    d_keys.alloc(N, nullptr);
    P->perm.alloc(N, cnt);
    tree_sort_points(P->x64.p, N, P->lo, scale20, d_keys.p, P->perm.p, st);
    std::vector<uint64_t> skeys(N);
    HFMM_CUDA(cudaMemcpyAsync(skeys.data(), d_keys.p, sizeof(uint64_t) * N, cudaMemcpyDeviceToHost, st));
    HFMM_CUDA(cudaStreamSynchronize(st));
    // The tree's boxes per level (sorted keys) and its leaves in Morton order.  Uniform: every
    // occupied cell down to the smallest depth whose fullest cell holds <= leaf_max points;
    // adaptive: a box is split only while it holds more than leaf_max points.
    std::vector<HostLevel> lv;
    std::vector<int32_t> w_ptr, w_idx, w_leaf;  // adaptive W lists (per leaf: box index, owner leaf)
    std::vector<int4> w_c2;                      // W boxes: centre in half level-L sides, level
    std::vector<uint64_t> leaf_key;
    std::vector<int32_t> leaf_lev, leaf_box, leaf_start;
    int L = 0;
    if (!cfg.adaptive) {
        L = cfg.depth;
        if (L <= 0) {
            for (L = 0; L < LMAX; ++L) {
                int sh = 3 * (LMAX - L);
                int64_t run = 0, best = 0;
                for (int64_t i = 0; i < N; ++i) {
                    run = (i > 0 && (skeys[i] >> sh) == (skeys[i - 1] >> sh)) ? run + 1 : 1;
                    best = std::max(best, run);
                }
                if (best <= cfg.leaf_max) break;
            }
        }
        L = std::min(L, LMAX);
        lv.resize(L + 1);
        for (int l = 0; l <= L; ++l) lv[l] = occupied_cells(skeys, l);
        leaf_key = lv[L].key;
        leaf_start = lv[L].start;
        leaf_lev.assign(leaf_key.size(), L);
        leaf_box.resize(leaf_key.size());
        std::iota(leaf_box.begin(), leaf_box.end(), 0);
    } else {
        const int maxdepth = cfg.depth > 0 ? std::min(cfg.depth, LMAX) : LMAX;
        lv.resize(maxdepth + 1);
        // depth first in Morton order, so each level's boxes come out with ascending keys
        struct Node {
            int l;
            int32_t b, e;
        };
        std::vector<Node> stack{{0, 0, (int32_t)N}};
        std::vector<Node> ch;
        while (!stack.empty()) {
            const Node nd = stack.back();
            stack.pop_back();
            const int sh = 3 * (LMAX - nd.l);
            HostLevel& h = lv[nd.l];
            h.key.push_back(skeys[nd.b] >> sh);
            h.start.push_back(nd.b);
            h.end.push_back(nd.e);
            if (nd.e - nd.b <= cfg.leaf_max || nd.l == maxdepth) {
                h.leaf.push_back((int32_t)leaf_key.size());
                leaf_key.push_back(skeys[nd.b] >> sh);
                leaf_lev.push_back(nd.l);
                leaf_box.push_back((int32_t)h.key.size() - 1);
                leaf_start.push_back(nd.b);
                L = std::max(L, nd.l);
            } else {
                h.leaf.push_back(-1);
                const int shc = 3 * (LMAX - nd.l - 1);
                ch.clear();
                for (int32_t i = nd.b; i < nd.e;) {
                    int32_t j = i;
                    while (j < nd.e && (skeys[j] >> shc) == (skeys[i] >> shc)) ++j;
                    ch.push_back({nd.l + 1, i, j});
                    i = j;
                }
                for (auto it = ch.rbegin(); it != ch.rend(); ++it) stack.push_back(*it);
            }
        }
        leaf_start.push_back((int32_t)N);
        lv.resize(L + 1);
    }
    P->L = L;
    P->adaptive = cfg.adaptive != 0;
    for (int l = 0; l <= L; ++l) {
        P->lev[l].nbox = (int64_t)lv[l].key.size();
        P->lev[l].side = D / std::ldexp(1.0, l);
        if (l >= 2) {
            P->lev[l].p = level_order(cfg, k, P->lev[l].side);
            if (P->lev[l].p > HFMM_PMAX) throw HfmmError{HFMM_E_INVALID, "expansion order above HFMM_PMAX"};
            P->lev[l].P = (P->lev[l].p + 1) * (P->lev[l].p + 1);
        }
        P->lev[l].s = std::min(1.0, k * 0.5 * std::sqrt(3.0) * P->lev[l].side);
    }
    // ---------------------------------------------------------- sorted point data
    const int64_t nleaf = (int64_t)leaf_key.size();
    P->nleaf = nleaf;
    const double sideL = P->lev[L].side;
    int lmin = L;  // coarsest leaf level
    for (int32_t l : leaf_lev) lmin = std::min(lmin, (int)l);
    P->leaf_levels.clear();
    for (int l = std::max(lmin, 2); l <= L; ++l)
        if (std::find(leaf_lev.begin(), leaf_lev.end(), l) != leaf_lev.end()) P->leaf_levels.push_back(l);
    // leaf centres in units of half a level-L side
    std::vector<int4> leaf_c2(nleaf);
    for (int64_t b = 0; b < nleaf; ++b) {
        int64_t c[3];
        demorton_h(leaf_key[b], c);
        const int sh = L - leaf_lev[b];
        leaf_c2[b] = make_int4((int)((2 * c[0] + 1) << sh), (int)((2 * c[1] + 1) << sh), (int)((2 * c[2] + 1) << sh),
                               leaf_lev[b]);
    }
    upload_legendre_tables();
    matvec_kernels_init();
    m2l_tc_init();
    P->p2p_variant = cfg.p2p_kernel >= 0 ? cfg.p2p_kernel : kDefaultP2PKernel;
    P->mv_mode = cfg.overlap >= 0 ? cfg.overlap : kDefaultOverlap;
    P->m2l_variant = cfg.m2l_kernel >= 0 ? cfg.m2l_kernel : kDefaultM2LKernel;
    m2l_ts_init();
    DBuf<double> d_w, d_x64s, d_w64s, d_V;
    DBuf<int32_t> d_t, d_tri, d_F, d_sstart;
    DBuf<uint64_t> d_leafkey, d_skey;
    DBuf<int4> d_pt_ijk;
    d_w.upload(W, nullptr, st);
    d_t.upload(T, nullptr, st);
    P->leaf_start.upload(leaf_start, cnt, st);
    P->leaf_ijk.upload(leaf_c2, cnt, st);
    P->pts.alloc(N, cnt);
    P->iperm.alloc(N, cnt);
    P->wscale.alloc(N, cnt);
    P->pt_leaf.alloc(N, cnt);
    d_x64s.alloc(3 * N, nullptr);
    d_w64s.alloc(N, nullptr);
    d_tri.alloc(N, nullptr);
    d_pt_ijk.alloc(N, nullptr);
    LeafData ld{P->pts.p, P->wscale.p, P->pt_leaf.p, d_pt_ijk.p, d_x64s.p, d_w64s.p, d_tri.p, P->iperm.p};
    tree_leaf_data(P->x64.p, d_w.p, d_t.p, P->perm.p, d_keys.p, L, P->leaf_ijk.p, P->leaf_start.p, nleaf, N, P->lo,
                   0.5 * sideL, k, ld, st);
    // near lists (self included) and target tiles
    std::vector<int32_t> nbr_ptr;
    std::vector<int64_t> hood;
    if (!P->adaptive) {  // 27 same-level boxes, on the device
        d_leafkey.upload(leaf_key, nullptr, st);
        tree_leaf_neighbours(d_leafkey.p, P->leaf_start.p, nleaf, L, P->nbr_ptr, P->nbr, nbr_ptr, hood, cnt, st);
        P->p2p_maxnbr = 27;
    } else {
        // Adaptive lists of leaf t (the interaction lists of Sec. 2.3 read for leaves at
        // several depths):
        //   U: every leaf that touches t, at any level: direct;
        //   W: the boxes under a split same-level neighbour of t that do not touch t while
        //      their parents do: their multipoles are evaluated at t's points (M2P) and t's
        //      points enter their local expansions (P2L, the dual list);
        // every other pair meets through M2L between same-level boxes that do not touch and
        // whose parents do.  A W box holding no more points than its expansion has terms is
        // cheaper summed directly, both ways: its leaves join U(t) and t joins theirs.  W boxes
        // need orders <= kWMaxP (the FP32 singular radial recurrence stays in range); a tree
        // that would need more is refused.
        constexpr int kWMaxP = 30;
        bool w_order_ok = true;
        auto touches = [&](int l1, uint64_t k1, int l2, uint64_t k2) {
            int64_t a[3], b[3];
            demorton_h(k1, a);
            demorton_h(k2, b);
            const int s1 = L - l1, s2 = L - l2;
            for (int d = 0; d < 3; ++d)
                if ((a[d] << s1) > ((b[d] + 1) << s2) || (b[d] << s2) > ((a[d] + 1) << s1)) return false;
            return true;
        };
        auto children = [&](int l, int64_t q, int64_t& c0, int64_t& c1) {
            const auto& kk = lv[l + 1].key;
            c0 = std::lower_bound(kk.begin(), kk.end(), lv[l].key[q] << 3) - kk.begin();
            c1 = std::lower_bound(kk.begin(), kk.end(), (lv[l].key[q] + 1) << 3) - kk.begin();
        };
        std::vector<int32_t> nbr;
        nbr_ptr.assign(nleaf + 1, 0);
        hood.assign(nleaf, 0);
        w_ptr.assign(nleaf + 1, 0);
        int maxn = 0;
        std::vector<std::pair<int, int64_t>> stack;
        std::vector<std::pair<int32_t, int32_t>> rev;  // (target leaf, source leaf) added from the source's side
        for (int64_t t = 0; t < nleaf; ++t) {
            const int lt = leaf_lev[t];
            const uint64_t kt = leaf_key[t];
            const size_t n0 = nbr.size();
            for (int m = 0; m <= lt; ++m) {
                int64_t c[3];
                demorton_h(kt >> (3 * (lt - m)), c);
                const int64_t nl = (int64_t)1 << m;
                for (int dx = -1; dx <= 1; ++dx)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dz = -1; dz <= 1; ++dz) {
                            const int64_t x = c[0] + dx, y = c[1] + dy, z = c[2] + dz;
                            if (x < 0 || y < 0 || z < 0 || x >= nl || y >= nl || z >= nl) continue;
                            const int64_t q = find_sorted(lv[m].key, morton_h(x, y, z));
                            if (q < 0) continue;
                            if (lv[m].leaf[q] >= 0) {
                                if (m == lt || touches(m, lv[m].key[q], lt, kt)) nbr.push_back(lv[m].leaf[q]);
                            } else if (m == lt) {
                                stack.assign(1, {m, q});
                                while (!stack.empty()) {
                                    const auto [l, bq] = stack.back();
                                    stack.pop_back();
                                    int64_t c0, c1;
                                    children(l, bq, c0, c1);
                                    for (int64_t cq = c0; cq < c1; ++cq) {
                                        const bool tch = touches(l + 1, lv[l + 1].key[cq], lt, kt);
                                        const int64_t npts = lv[l + 1].end[cq] - lv[l + 1].start[cq];
                                        if (!tch && npts <= P->lev[l + 1].P) {  // small W box: direct
                                            const int64_t l0 = std::lower_bound(leaf_start.begin(), leaf_start.end() - 1,
                                                                                lv[l + 1].start[cq]) - leaf_start.begin();
                                            const int64_t l1 = std::lower_bound(leaf_start.begin(), leaf_start.end() - 1,
                                                                                lv[l + 1].end[cq]) - leaf_start.begin();
                                            for (int64_t s2 = l0; s2 < l1; ++s2) {
                                                nbr.push_back((int32_t)s2);
                                                rev.push_back({(int32_t)s2, (int32_t)t});
                                            }
                                        } else if (!tch) {  // boxes of level >= 2 here: level-1 boxes all touch
                                            w_order_ok = w_order_ok && P->lev[l + 1].p <= kWMaxP;
                                            int64_t cc[3];
                                            demorton_h(lv[l + 1].key[cq], cc);
                                            const int sh = L - (l + 1);
                                            w_c2.push_back(make_int4((int)((2 * cc[0] + 1) << sh), (int)((2 * cc[1] + 1) << sh),
                                                                     (int)((2 * cc[2] + 1) << sh), l + 1));
                                            w_idx.push_back((int32_t)cq);
                                            w_leaf.push_back((int32_t)t);
                                        } else if (lv[l + 1].leaf[cq] >= 0) {
                                            nbr.push_back(lv[l + 1].leaf[cq]);
                                        } else {
                                            stack.push_back({l + 1, cq});
                                        }
                                    }
                                }
                            }
                        }
            }
            nbr_ptr[t + 1] = (int32_t)nbr.size();
            w_ptr[t + 1] = (int32_t)w_idx.size();
        }
        {  // merge the pairs added from the source's side into the targets' lists
            std::stable_sort(rev.begin(), rev.end(),
                             [](const std::pair<int32_t, int32_t>& a, const std::pair<int32_t, int32_t>& b) {
                                 return a.first < b.first;
                             });
            std::vector<int32_t> merged, mptr(nleaf + 1, 0);
            merged.reserve(nbr.size() + rev.size());
            size_t r = 0;
            for (int64_t t = 0; t < nleaf; ++t) {
                merged.insert(merged.end(), nbr.begin() + nbr_ptr[t], nbr.begin() + nbr_ptr[t + 1]);
                for (; r < rev.size() && rev[r].first == t; ++r) merged.push_back(rev[r].second);
                mptr[t + 1] = (int32_t)merged.size();
            }
            nbr.swap(merged);
            nbr_ptr.swap(mptr);
            for (int64_t t = 0; t < nleaf; ++t) {
                for (int32_t q = nbr_ptr[t]; q < nbr_ptr[t + 1]; ++q) hood[t] += leaf_start[nbr[q] + 1] - leaf_start[nbr[q]];
                maxn = std::max(maxn, nbr_ptr[t + 1] - nbr_ptr[t]);
            }
        }
        if (!w_order_ok)
            throw HfmmError{HFMM_E_INVALID, "adaptive tree: leaves of different depths meet where the expansion "
                                            "order exceeds 30; use the uniform tree (adaptive = 0)"};
        P->nbr_ptr.upload(nbr_ptr, cnt, st);
        P->nbr.upload(nbr, cnt, st);
        P->p2p_maxnbr = maxn;
        P->leaf_lev.upload(leaf_lev, cnt, st);
        P->leaf_box.upload(leaf_box, cnt, st);
    }
    std::vector<int4> tiles;
    for (int64_t b = 0; b < nleaf; ++b)
        for (int32_t i0 = leaf_start[b]; i0 < leaf_start[b + 1]; i0 += kP2PTile)
            tiles.push_back(make_int4((int)b, i0, std::min(kP2PTile, leaf_start[b + 1] - i0), 0));
    P->ntiles = (int64_t)tiles.size();
    double pairs = 0.0;
    int64_t cap = 0;
    for (int64_t b = 0; b < nleaf; ++b) {
        pairs += (double)(leaf_start[b + 1] - leaf_start[b]) * (double)hood[b];
        cap = std::max(cap, hood[b]);
    }
    P->cost[0] = pairs - (double)N;
    P->p2p_cap = (int)std::min<int64_t>(cap, 1 << 30);
    P->cost[4] = (double)N;
    P->p2p_shift = (float)(0.5 * k * sideL);
    // direct pairs are at most 2 sqrt(3) coarsest-leaf sides apart
    const double side_c = P->lev[lmin].side;
    P->poly_p2p = 12.0 * (k * side_c) * (k * side_c) * 1.001 <= (double)HFMM_POLY_UMAX;
    HFMM_CUDA(cudaStreamSynchronize(st));
    d_keys.release();

    P->tiles.upload(tiles, cnt, st);
    P->sig.alloc(N, cnt);
    P->phi.alloc(N, cnt);
    P->dev_err.alloc(1, cnt);
    HFMM_CUDA(cudaMemsetAsync(P->dev_err.p, 0, sizeof(int), st));
    P->host_x = X;
    P->host_w = W;
    P->host_t = T;

    // ---------------------------------------------------------- far field (Sec. 2.3)
    P->m2m_items_begin.assign(L + 2, 0);
    P->m2m_items_end.assign(L + 2, 0);
    P->l2l_items_begin.assign(L + 2, 0);
    P->l2l_items_end.assign(L + 2, 0);
    if (L >= 2) {
        int64_t off = 0;
        for (int l = 2; l <= L; ++l) {
            P->lev[l].mofs = off;
            off += (P->lev[l].nbox * P->lev[l].P + 15) & ~15ll;  // 128-byte aligned level blocks
        }
        P->coef_m_total = off;
        for (int l = 2; l <= L; ++l) {
            P->lev[l].lofs = off;
            off += (P->lev[l].nbox * P->lev[l].P + 15) & ~15ll;
        }
        P->coef_total = off;
        P->cost[5] = (double)off;
        // tree-pass byte model: leaf-level coefficients (P2M writes, L2P reads), level-2 and
        // all-level multipole coefficients (M2M / L2L read one side and write the other)
        for (int32_t l : leaf_lev)
            if (l >= 2) P->cost[8] += (double)P->lev[l].P;
        P->cost[9] = (double)(P->lev[2].nbox * P->lev[2].P);
        for (int l = 2; l <= L; ++l) P->cost[10] += (double)(P->lev[l].nbox * P->lev[l].P);
        P->cost[11] = (double)(P->lev[L].nbox * P->lev[L].P);
        if (P->adaptive) {
            std::vector<AdLevel> al(L + 1);
            for (int l = 2; l <= L; ++l) al[l] = AdLevel{P->lev[l].mofs, P->lev[l].lofs, P->lev[l].p, (float)P->lev[l].s};
            P->ad_lev.upload(al, cnt, st);
            P->w_ptr.upload(w_ptr, cnt, st);
            P->w_idx.upload(w_idx, cnt, st);
            P->w_leaf.upload(w_leaf, cnt, st);
            P->w_c2.upload(w_c2, cnt, st);
            P->n_w = (int64_t)w_idx.size();
            for (const int4& c : w_c2) P->w_maxP = std::max(P->w_maxP, P->lev[c.w].P);
        }
        int64_t ooff = 0;
        for (int l = 2; l <= L; ++l) {
            int Pl = P->lev[l].P;
            P->lev[l].m2l_op = ooff;
            ooff += 316ll * Pl * Pl;
            if (l >= 3) {
                int Pp = P->lev[l - 1].P;
                P->lev[l].pc_op = ooff;
                ooff += 8ll * Pl * Pp;
                P->lev[l].m2m_op = ooff;
                ooff += 8ll * Pl * Pp;
            }
        }
        if (cfg.mem_budget_bytes > 0 &&
            (double)P->dev_bytes + 8.0 * (double)(ooff + P->coef_total) > cfg.mem_budget_bytes)
            throw HfmmError{HFMM_E_NOMEM, "plan exceeds the configured device memory budget"};
        P->coef.alloc(P->coef_total, cnt);
        P->ops.alloc(ooff, cnt);
        // offset table: 343 offsets in [-3,3]^3 minus the 27 neighbours -> 316 slots
        int slot[343];
        std::vector<double> d0_unit;
        int ns = 0;
        for (int o = 0; o < 343; ++o) {
            int dx = o / 49 - 3, dy = (o / 7) % 7 - 3, dz = o % 7 - 3;
            if (std::abs(dx) <= 1 && std::abs(dy) <= 1 && std::abs(dz) <= 1) {
                slot[o] = -1;
                continue;
            }
            slot[o] = ns++;
            d0_unit.push_back(dx);
            d0_unit.push_back(dy);
            d0_unit.push_back(dz);
        }
        // canonical offsets (non-negative components) and each slot's reflections of one
        std::vector<double> canon_unit;
        std::vector<int4> refl(316);
        {
            int cidx[64];
            for (int q = 0; q < 64; ++q) cidx[q] = -1;
            int nc = 0;
            for (int q = 0; q < 316; ++q) {
                const int dx = (int)d0_unit[3 * q], dy = (int)d0_unit[3 * q + 1], dz = (int)d0_unit[3 * q + 2];
                const int key = std::abs(dx) * 16 + std::abs(dy) * 4 + std::abs(dz);
                if (cidx[key] < 0) {
                    cidx[key] = nc++;
                    canon_unit.push_back(std::abs(dx));
                    canon_unit.push_back(std::abs(dy));
                    canon_unit.push_back(std::abs(dz));
                }
                refl[q] = make_int4(cidx[key], dx < 0, dy < 0, dz < 0);
            }
        }
        const int ncanon = (int)(canon_unit.size() / 3);
        DBuf<int4> d_refl;
        d_refl.upload(refl, nullptr, st);
        // the canonical operators of the tensor-core levels stay resident (target-stationary M2L)
        {
            int64_t coff = 0;
            for (int l = 2; l <= L; ++l)
                if (cfg.m2l_tensor && P->lev[l].P <= 64) {
                    P->lev[l].canon_op = coff;
                    coff += (int64_t)ncanon * kTsOpElems;  // packed BF16 (m2l_ts.cu)
                }
            if (coff > 0) P->m2l_canon.alloc((size_t)coff, cnt);
        }
        for (int l = 2; l <= L; ++l) {
            const LevelInfo& li = P->lev[l];
            double a = 0.5 * std::sqrt(3.0) * li.side;
            ProjectionJob job{};
            job.type = 1;
            job.pf = job.pb = li.p;
            job.sf = job.sb = li.s;
            job.rho = choose_rho(k, a, li.p);
            job.nth = job.pb + (job.pf + 1) / 2 + 16;
            job.nph = 2 * job.nth + 2;
            job.nops = ncanon;
            std::vector<double> d0(canon_unit);
            for (double& v : d0) v *= li.side;  // c_source - c_target
            job.d0 = d0.data();
            DBuf<float2> canon;
            canon.alloc((size_t)ncanon * li.P * li.P, nullptr);
            job.out = canon.p;
            job.out2 = nullptr;
            build_projection_ops(job, k, st);
            expand_m2l_reflections(canon.p, li.P, 316, d_refl.p, P->ops.p + li.m2l_op, st);
            if (li.canon_op >= 0) m2l_ts_pack_ops(canon.p, li.P, ncanon, P->m2l_canon.p + li.canon_op, st);
            HFMM_CUDA(cudaStreamSynchronize(st));  // canon is freed at the end of this scope
            if (l >= 3) {
                const LevelInfo& lp = P->lev[l - 1];
                ProjectionJob pj{};
                pj.type = 0;
                pj.pf = lp.p;
                pj.sf = lp.s;
                pj.pb = li.p;
                pj.sb = li.s;
                pj.rho = choose_rho(k, a, li.p);
                pj.nth = pj.pb + (pj.pf + 1) / 2 + 16;
                pj.nph = 2 * pj.nth + 2;
                pj.nops = 8;
                std::vector<double> dd(24);
                for (int o = 0; o < 8; ++o) {
                    int bits[3] = {(o >> 2) & 1, (o >> 1) & 1, o & 1};
                    for (int d = 0; d < 3; ++d) dd[3 * o + d] = -0.25 * lp.side * (2.0 * bits[d] - 1.0);  // c_parent - c_child
                }
                pj.d0 = dd.data();
                pj.out = P->ops.p + li.pc_op;
                pj.out2 = P->ops.p + li.m2m_op;
                build_projection_ops(pj, k, st);
            }
        }
        {
            // FP32 translation operators: at high orders on small boxes (k a well below p) the
            // outgoing functions exceed FP32's range; such a plan would return NaN
            DBuf<int> bad;
            bad.alloc(1, nullptr);
            HFMM_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
            k_flag_nonfinite<<<(unsigned)std::min<int64_t>((ooff + 255) / 256, 65535), 256, 0, st>>>(P->ops.p, ooff,
                                                                                                 bad.p);
            HFMM_CUDA(cudaGetLastError());
            int h_bad = 0;
            HFMM_CUDA(cudaMemcpyAsync(&h_bad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
            HFMM_CUDA(cudaStreamSynchronize(st));
            if (h_bad)
                throw HfmmError{HFMM_E_INVALID,
                                "translation operators overflow FP32 at this expansion order and box size: "
                                "lower p_fixed / p_min"};
        }
        // work items
        std::vector<TransItem> items;
        std::vector<int2> cols;
        for (int l = L - 1; l >= 2; --l) {  // M2M: children at l+1 -> parents at l
            std::vector<std::vector<int2>> b8(8);
            const HostLevel& ch = lv[l + 1];
            for (int64_t c = 0; c < (int64_t)ch.key.size(); ++c) {
                int64_t par = find_sorted(lv[l].key, ch.key[c] >> 3);
                b8[ch.key[c] & 7].push_back(make_int2((int)c, (int)par));
            }
            const PairBuckets pb = PairBuckets::from(b8);
            std::vector<int64_t> ops(8);
            for (int o = 0; o < 8; ++o) ops[o] = P->lev[l + 1].m2m_op + (int64_t)o * P->lev[l].P * P->lev[l + 1].P;
            P->m2m_items_begin[l] = (int64_t)items.size();
            emit_items(pb, ops, P->lev[l + 1].mofs, P->lev[l].mofs, P->lev[l + 1].P, P->lev[l].P, 1, items, cols);
            P->m2m_items_end[l] = (int64_t)items.size();
            P->cost[2] += (double)ch.key.size() * P->lev[l].P * P->lev[l + 1].P;
        }
        P->m2l_items_begin = (int64_t)items.size();
        int64_t m2l_count = 0;
        std::vector<int64_t> lev_item_b(L + 1, 0), lev_item_e(L + 1, 0);
        std::vector<int> lev_width(L + 1, HFMM_TRANS_NB);
        std::vector<int64_t> lev_pairs(L + 1, 0);
        std::vector<int16_t> slot16(slot, slot + 343);
        DBuf<int16_t> d_slot;
        d_slot.upload(slot16, nullptr, st);
        std::vector<TsTile> ts_tiles;
        std::vector<TsChunk> ts_chunks;
        std::vector<int2> ts_cols;
        // tile size of the target-stationary M2L: the largest of 128, 64, 32 targets that still
        // gives every SM a tile (one block per SM at a time; larger tiles fill the chunks better)
        int ts_tt = 32;
        std::vector<int64_t> ts_bxofs(L + 1, -1);
        {
            int dev = 0, nsm = 1;
            HFMM_CUDA(cudaGetDevice(&dev));
            HFMM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
            for (int tt = kTsTile; tt >= 32; tt /= 2) {
                int64_t tiles = 0;
                for (int l = 2; l <= L; ++l)
                    if (P->lev[l].canon_op >= 0) tiles += ((int64_t)lv[l].key.size() + tt - 1) / tt;
                if (tiles >= (int64_t)nsm) {
                    ts_tt = tt;
                    break;
                }
            }
            // the split multipoles of the tensor-core levels, 64 x 16 bytes per box
            P->ts_split = TsSplitTable{};
            P->ts_split_boxes = 0;
            for (int l = 2; l <= L; ++l)
                if (P->lev[l].canon_op >= 0 && P->ts_split.nlev < kTsMaxLevels &&
                    lv[l].key.size() < ((size_t)1 << 24)) {  // column entries hold 24-bit box indices
                    TsSplitLevel& e = P->ts_split.lev[P->ts_split.nlev++];
                    e.src = P->lev[l].mofs;
                    e.bx = P->ts_split_boxes * 64;
                    e.P = P->lev[l].P;
                    e.nbox = (int32_t)lv[l].key.size();
                    ts_bxofs[l] = e.bx;
                    P->ts_split_boxes += e.nbox;
                }
        }
        for (int l = 2; l <= L; ++l) {
            lev_item_b[l] = (int64_t)items.size();
            // interaction lists (children of the parent's neighbours that are not
            // neighbours), built on the device and bucketed by offset slot
            PairBuckets pb;
            DBuf<uint64_t> d_lkey;
            d_lkey.upload(lv[l].key, nullptr, st);
            const int64_t npair = tree_m2l_lists(d_lkey.p, (int64_t)lv[l].key.size(), l, d_slot.p, pb.pairs, pb.start, st);
            m2l_count += npair;
            lev_pairs[l] = npair;
            P->cost[1] += (double)npair * P->lev[l].P * P->lev[l].P;
            std::vector<int64_t> ops(316);
            for (int o = 0; o < 316; ++o) ops[o] = P->lev[l].m2l_op + (int64_t)o * P->lev[l].P * P->lev[l].P;
            // SIMT levels with few targets per offset (the coarse ones) take narrow items
            int width = HFMM_TRANS_NB;
            if (!(cfg.m2l_tensor && P->lev[l].P <= 64)) {
                int64_t busy = 0, pairs = 0;
                for (size_t g = 0; g + 1 < pb.start.size(); ++g) {
                    busy += pb.size(g) > 0;
                    pairs += pb.size(g);
                }
                const int64_t mean = busy ? pairs / busy : 0;
                // measured on the 1.97 M-point workload: 16 columns beat 8 at a mean of 11
                // (order-16 level) and beat 64 at a mean of 39 (order-10 level)
                width = mean <= 6 ? 8 : mean <= 48 ? 16 : HFMM_TRANS_NB;
            }
            lev_width[l] = width;
            if (ts_bxofs[l] >= 0)
                emit_ts_level(pb, refl, ncanon, (int64_t)lv[l].key.size(), P->lev[l].P, ts_bxofs[l], P->lev[l].lofs,
                              P->lev[l].canon_op, ts_tt, ts_tiles, ts_chunks, ts_cols);
            emit_items(pb, ops, P->lev[l].mofs, P->lev[l].lofs, P->lev[l].P, P->lev[l].P, 1, items, cols, width);
            lev_item_e[l] = (int64_t)items.size();
        }
        P->m2l_items_end = (int64_t)items.size();
        P->m2l_count = m2l_count;
        if (!ts_tiles.empty()) {
            // longest tiles first, so that the last wave is short
            std::vector<int64_t> work(ts_tiles.size());
            for (size_t t = 0; t < ts_tiles.size(); ++t) {
                int64_t n = 0;
                for (int c = 0; c < ts_tiles[t].nchunk; ++c) n += ts_chunks[(size_t)(ts_tiles[t].chunk0 + c)].ncol;
                work[t] = n;
            }
            std::vector<size_t> order(ts_tiles.size());
            for (size_t t = 0; t < order.size(); ++t) order[t] = t;
            std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return work[a] > work[b]; });
            std::vector<TsTile> sorted;
            sorted.reserve(order.size());
            for (size_t t : order) {
                sorted.push_back(ts_tiles[t]);
                P->ts_max_chunks = std::max(P->ts_max_chunks, ts_tiles[t].nchunk);
            }
            P->ts_tiles.upload(sorted, cnt, st);
            P->ts_chunks.upload(ts_chunks, cnt, st);
            P->ts_cols.upload(ts_cols, cnt, st);
            P->ts_bx.alloc((size_t)P->ts_split_boxes * 64, cnt);
            P->n_ts_tiles = (int64_t)sorted.size();
            int optin = 0, dev = 0;
            HFMM_CUDA(cudaGetDevice(&dev));
            HFMM_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
            bool all_levels = true;  // every tensor-core level must be in the tiles
            for (int l = 2; l <= L; ++l) all_levels &= P->lev[l].canon_op < 0 || ts_bxofs[l] >= 0;
            if (!all_levels || m2l_ts_smem(P->ts_max_chunks) > (size_t)optin) {
                // a tile with more chunks than fit beside its locals: keep the source-stationary kernel
                P->n_ts_tiles = 0;
            }
        }
        for (int l = 3; l <= L; ++l) {  // L2L: parents at l-1 -> children at l
            std::vector<std::vector<int2>> b8(8);
            const HostLevel& ch = lv[l];
            for (int64_t c = 0; c < (int64_t)ch.key.size(); ++c) {
                int64_t par = find_sorted(lv[l - 1].key, ch.key[c] >> 3);
                b8[ch.key[c] & 7].push_back(make_int2((int)par, (int)c));
            }
            const PairBuckets pb = PairBuckets::from(b8);
            std::vector<int64_t> ops(8);
            for (int o = 0; o < 8; ++o) ops[o] = P->lev[l].pc_op + (int64_t)o * P->lev[l].P * P->lev[l - 1].P;
            P->l2l_items_begin[l] = (int64_t)items.size();
            // accumulating (a child has one parent, but the SIMT kernel splits a coarse level's
            // K across blocks, whose partial sums meet in the child's locals)
            emit_items(pb, ops, P->lev[l - 1].lofs, P->lev[l].lofs, P->lev[l - 1].P, P->lev[l].P, 1, items, cols);
            P->l2l_items_end[l] = (int64_t)items.size();
            P->cost[2] += (double)ch.key.size() * P->lev[l].P * P->lev[l - 1].P;
        }
        // Tensor-core translations: M2L of levels with (p+1)^2 <= 64, and M2M / L2L between
        // two such levels of equal order.  Operators are packed once; items of one operator
        // are grouped (consecutive in the item list) for one block each.
        std::vector<int4> groups;
        std::vector<std::pair<int64_t, int64_t>> pack;  // (fp32 operator offset, count) per packed block
        std::vector<int> pack_P;
        int64_t tc_ops = 0;
        auto tc_level = [&](int l) { return cfg.m2l_tensor && P->lev[l].P <= 64; };
        std::vector<int64_t> m2l_base(L + 2, -1), m2m_base(L + 2, -1), l2l_base(L + 2, -1);
        for (int l = 2; l <= L; ++l) {
            if (tc_level(l)) {
                m2l_base[l] = tc_ops;
                pack.push_back({P->lev[l].m2l_op, 316});
                pack_P.push_back(P->lev[l].P);
                tc_ops += 316;
            }
            if (l <= L - 1 && tc_level(l) && tc_level(l + 1) && P->lev[l].P == P->lev[l + 1].P) {
                m2m_base[l] = tc_ops;  // parents at l
                pack.push_back({P->lev[l + 1].m2m_op, 8});
                pack_P.push_back(P->lev[l].P);
                tc_ops += 8;
            }
            if (l >= 3 && tc_level(l) && tc_level(l - 1) && P->lev[l].P == P->lev[l - 1].P) {
                l2l_base[l] = tc_ops;  // children at l
                pack.push_back({P->lev[l].pc_op, 8});
                pack_P.push_back(P->lev[l].P);
                tc_ops += 8;
            }
        }
        if (tc_ops > 0) {
            P->aops.alloc((size_t)tc_ops * m2l_tc_op_elems(), cnt);
            int64_t at = 0;
            for (size_t q = 0; q < pack.size(); ++q) {
                m2l_tc_pack(P->ops.p + pack[q].first, pack_P[q], (int)pack[q].second,
                            P->aops.p + (size_t)at * m2l_tc_op_elems(), st);
                at += pack[q].second;
            }
        }
        const int kGroupItems = m2l_tc_max_group();  // split further by apply_tc_group
        const int kSmallGroup = 4;  // M2M/L2L have 8 operators per level: small groups keep every SM busy
        auto make_groups = [&](int64_t ib, int64_t ie, int64_t op0, int64_t opsz, int64_t base, int Pl,
                               int gmax) {
            for (int64_t b = ib; b < ie;) {
                int64_t e = b;
                while (e < ie && e - b < gmax && items[e].op == items[b].op) ++e;
                groups.push_back(make_int4((int)b, (int)(e - b), (int)(base + (items[b].op - op0) / opsz), Pl));
                b = e;
            }
        };
        for (int l = 2; l <= L; ++l) {
            if (m2l_base[l] >= 0) {
                P->cost[6] += (double)lev_pairs[l] * P->lev[l].P * P->lev[l].P;
                P->cost[7] += (double)lev_pairs[l];
            }
            if (m2l_base[l] < 0) {
                auto& R = P->m2l_simt;
                if (!R.empty() && R.back().end == lev_item_b[l] && R.back().width == lev_width[l]) {
                    R.back().end = lev_item_e[l];
                    R.back().pout_max = std::max(R.back().pout_max, P->lev[l].P);
                } else {
                    R.push_back({lev_item_b[l], lev_item_e[l], P->lev[l].P, lev_width[l]});
                }
                continue;
            }
            make_groups(lev_item_b[l], lev_item_e[l], P->lev[l].m2l_op, (int64_t)P->lev[l].P * P->lev[l].P,
                        m2l_base[l], P->lev[l].P, kGroupItems);
        }
        P->n_tc_groups = (int64_t)groups.size();  // M2L groups come first
        P->m2m_tc.assign(L + 2, {0, 0});
        P->l2l_tc.assign(L + 2, {0, 0});
        for (int l = 2; l <= L; ++l) {
            if (m2m_base[l] >= 0) {
                int64_t g0 = (int64_t)groups.size();
                make_groups(P->m2m_items_begin[l], P->m2m_items_end[l], P->lev[l + 1].m2m_op,
                            (int64_t)P->lev[l].P * P->lev[l + 1].P, m2m_base[l], P->lev[l].P, kSmallGroup);
                P->m2m_tc[l] = {g0, (int64_t)groups.size()};
            }
            if (l2l_base[l] >= 0) {
                int64_t g0 = (int64_t)groups.size();
                make_groups(P->l2l_items_begin[l], P->l2l_items_end[l], P->lev[l].pc_op,
                            (int64_t)P->lev[l].P * P->lev[l - 1].P, l2l_base[l], P->lev[l].P, kSmallGroup);
                P->l2l_tc[l] = {g0, (int64_t)groups.size()};
            }
        }
        P->tc_groups.upload(groups, cnt, st);
        P->items.upload(items, cnt, st);
        P->item_cols.upload(cols, cnt, st);
        P->host_items = std::move(items);
        P->host_cols = std::move(cols);
        P->host_groups = std::move(groups);
        P->tc_m2l_base = P->n_tc_groups;
        P->m2m_tc_base = P->m2m_tc;
        P->l2l_tc_base = P->l2l_tc;
        apply_tc_group(P, cfg.tc_group > 0 ? cfg.tc_group : m2l_tc_max_group(), st);
    }

    // ---------------------------------------------------------- self / near correction (Sec. 2.2)
    int ls = L;
    while (ls > 0 && P->lev[ls].side < P->r_near) --ls;
    const HostLevel S = P->adaptive ? occupied_cells(skeys, ls) : lv[ls];
    std::vector<double> Vh(V, V + 3 * nv);
    std::vector<int32_t> Fh(F, F + 3 * nt);
    d_V.upload(Vh, nullptr, st);
    d_F.upload(Fh, nullptr, st);
    d_skey.upload(S.key, nullptr, st);
    d_sstart.upload(S.start, nullptr, st);
    CorrInputs ci{};
    ci.x64s = d_x64s.p;
    ci.tri_s = d_tri.p;
    ci.V = d_V.p;
    ci.F = d_F.p;
    ci.iperm = P->iperm.p;
    ci.w64s = d_w64s.p;
    ci.skey = d_skey.p;
    ci.sstart = d_sstart.p;
    ci.nsbox = (int64_t)S.key.size();
    ci.search_level = ls;
    ci.L = L;
    ci.pt_ijk = d_pt_ijk.p;
    ci.N = N;
    ci.k = k;
    ci.r_near = P->r_near;
    ci.quad_order = cfg.quad_order;
    P->corr_nnz = build_correction(P, ci, st);
    P->cost[3] = (double)P->corr_nnz;
    if (cfg.precision == 1) accurate_setup(P, st);
    HFMM_CUDA(cudaStreamSynchronize(st));
    if (cfg.mem_budget_bytes > 0 && (double)P->dev_bytes > cfg.mem_budget_bytes)
        throw HfmmError{HFMM_E_NOMEM, "plan exceeds the configured device memory budget"};
}

// =================================================================== C ABI
#define HFMM_GUARD_BEGIN try {
#define HFMM_GUARD_END                               \
    }                                                \
    catch (const HfmmError& e) {                     \
        g_last_error = e.what;                       \
        return e.code;                               \
    }                                                \
    catch (const std::bad_alloc&) {                  \
        g_last_error = "host allocation failed";     \
        return HFMM_E_NOMEM;                         \
    }                                                \
    catch (...) {                                    \
        g_last_error = "unexpected exception";       \
        return HFMM_E_CUDA;                          \
    }

extern "C" {

void hfmm_default_config(hfmm_config* c) {
    if (!c) return;
    c->leaf_max = 64;
    c->depth = 0;
    c->p_fixed = 0;
    c->p_min = 7;
    c->near_factor = 1.0;
    c->quad_order = 10;
    c->restart = 30;
    c->max_iter = 1000;
    c->tol = 1e-4;
    c->mem_budget_bytes = 0.0;
    c->m2l_tensor = 1;
    c->adaptive = 0;
    c->autotune = 0;
    c->p2p_kernel = -1;
    c->m2l_kernel = -1;
    c->tc_group = 0;
    c->overlap = -1;
    c->precision = 0;
}

const char* hfmm_last_error(void) { return g_last_error.c_str(); }

const char* hfmm_status_string(int s) {
    switch (s) {
        case HFMM_OK: return "ok";
        case HFMM_NOT_CONVERGED: return "GMRES did not reach the tolerance within max_iter";
        case HFMM_E_INVALID: return "invalid argument";
        case HFMM_E_MESH: return "degenerate or invalid mesh";
        case HFMM_E_NOMEM: return "out of device memory or over the memory budget";
        case HFMM_E_CUDA: return "CUDA runtime error";
        case HFMM_E_TIMEOUT: return "device wait timed out";
        case HFMM_E_OVERFLOW: return "fixed-capacity table overflowed";
        default: return "unknown status";
    }
}

int hfmm_plan_create(const hfmm_config* cfg, const double* vertices, int64_t n_vert, const int32_t* tris,
                     int64_t n_tri, double k_re, double k_im, void* stream, hfmm_plan** out) {
    if (out) *out = nullptr;
    if (!cfg || !vertices || !tris || !out || n_vert <= 0 || n_tri <= 0) return HFMM_E_INVALID;
    if (!(k_re > 0.0) || !std::isfinite(k_re) || k_im != 0.0) return HFMM_E_INVALID;
    if (cfg->leaf_max < 1 || cfg->depth < 0 || cfg->depth > 20 || cfg->p_fixed < 0 || cfg->p_fixed > HFMM_PMAX ||
        cfg->p_min < 0 || cfg->p_min > HFMM_PMAX || !(cfg->near_factor >= 0.0) || cfg->quad_order < 2 ||
        cfg->quad_order > 64 || cfg->restart < 1 || cfg->max_iter < 1 || !(cfg->tol > 0.0) ||
        (cfg->m2l_tensor != 0 && cfg->m2l_tensor != 1) || (cfg->adaptive != 0 && cfg->adaptive != 1) ||
        (cfg->autotune != 0 && cfg->autotune != 1) || cfg->p2p_kernel < -1 || cfg->p2p_kernel > 2 ||
        cfg->m2l_kernel < -1 || cfg->m2l_kernel > 1 ||
        (cfg->tc_group != 0 && cfg->tc_group != 8 && cfg->tc_group != 16 && cfg->tc_group != 32) ||
        cfg->overlap < -1 || cfg->overlap > 1 || (cfg->precision != 0 && cfg->precision != 1))
        return HFMM_E_INVALID;
    if (3 * n_tri > (int64_t)INT32_MAX / 2) return HFMM_E_INVALID;
    HFMM_GUARD_BEGIN
    std::unique_ptr<hfmm_plan> P(new hfmm_plan());
    P->cfg = *cfg;
    P->k = k_re;
    build_plan(P.get(), vertices, n_vert, tris, n_tri, (cudaStream_t)stream);
    if (cfg->autotune) tune_plan(P.get(), (cudaStream_t)stream);
    *out = P.release();
    return HFMM_OK;
    HFMM_GUARD_END
}

void hfmm_plan_destroy(hfmm_plan* P) {
    if (!P) return;
    // the plan's own streams (graph replays launch on the caller's streams, which the caller has
    // finished with before releasing the plan); no device-wide wait, so that other plans'
    // work in flight, or a graph capture on another thread, is not held up or invalidated
    if (P->mvg.cap) cudaStreamSynchronize(P->mvg.cap);
    if (P->mvg.side) cudaStreamSynchronize(P->mvg.side);
    if (P->batch.cap_stream) cudaStreamSynchronize(P->batch.cap_stream);
    delete P;
}

int64_t hfmm_num_points(const hfmm_plan* P) { return P ? P->N : -1; }

int hfmm_points(const hfmm_plan* P, double* xyz, double* w, int32_t* tri) {
    if (!P) return HFMM_E_INVALID;
    if (xyz) std::memcpy(xyz, P->host_x.data(), sizeof(double) * 3 * P->N);
    if (w) std::memcpy(w, P->host_w.data(), sizeof(double) * P->N);
    if (tri) std::memcpy(tri, P->host_t.data(), sizeof(int32_t) * P->N);
    return HFMM_OK;
}

int hfmm_plan_info(const hfmm_plan* P, int* depth, int* orders, int64_t* n_leaves, int64_t* corr_nnz,
                   int64_t* m2l_translations, int64_t* device_bytes) {
    if (!P) return HFMM_E_INVALID;
    if (depth) *depth = P->L;
    if (orders)
        for (int l = 0; l < 32; ++l) orders[l] = (l <= P->L) ? P->lev[l].p : 0;
    if (n_leaves) *n_leaves = P->nleaf;
    if (corr_nnz) *corr_nnz = P->corr_nnz;
    if (m2l_translations) *m2l_translations = P->m2l_count;
    if (device_bytes) *device_bytes = (int64_t)P->dev_bytes;
    return HFMM_OK;
}

int hfmm_matvec_parts(hfmm_plan* P, const void* density, void* potential, int nrhs, int parts, void* stream) {
    if (!P || !density || !potential || nrhs < 1 || parts < 0 || parts > 7) return HFMM_E_INVALID;
    HFMM_GUARD_BEGIN
    cudaStream_t st = (cudaStream_t)stream;
    for (int r0 = 0; r0 < nrhs;) {
        const int R = std::min(nrhs - r0, 64);
        const float2* d = (const float2*)density + (int64_t)r0 * P->N;
        float2* o = (float2*)potential + (int64_t)r0 * P->N;
        if (parts == 7 && R > 1 && batch_supported(P, R)) {
            batched_matvec(P, d, o, R, st);
            r0 += R;
            continue;
        }
        launch_density_prep(P, d, VecKind::Complex64, P->sig.p, st);
        run_matvec_sorted(P, parts, st);
        launch_output(P, P->phi.p, o, VecKind::Complex64, st);
        ++r0;
    }
    HFMM_CUDA(cudaGetLastError());
    return HFMM_OK;
    HFMM_GUARD_END
}

int hfmm_solve_group(hfmm_plan* const* plans, int G, const void* const* rhs, void* const* x_out, int* iters_out,
                     double* relres_out, void* stream) {
    if (!plans || !rhs || !x_out || G < 1 || G > HFMM_GROUP_MAX) return HFMM_E_INVALID;
    for (int g = 0; g < G; ++g) {
        if (!plans[g] || !rhs[g] || !x_out[g]) return HFMM_E_INVALID;
        for (int q = 0; q < g; ++q)
            if (plans[q] == plans[g]) {
                g_last_error = "hfmm_solve_group: a plan appears twice (each solve needs its own plan)";
                return HFMM_E_INVALID;
            }
    }
    HFMM_GUARD_BEGIN
    return run_gmres_group(plans, G, rhs, x_out, iters_out, relres_out, (cudaStream_t)stream);
    HFMM_GUARD_END
}

int hfmm_solver_info(const hfmm_plan* P, int* cycle_graph) {
    if (!P || !cycle_graph) return HFMM_E_INVALID;
    *cycle_graph = P->gm_used;
    return HFMM_OK;
}

int hfmm_matvec_df(hfmm_plan* P, const void* density_df, void* potential_df, int parts, void* stream) {
    if (!P || !density_df || !potential_df || parts < 0 || parts > 7) return HFMM_E_INVALID;
    if (P->cfg.precision != 1) {
        g_last_error = "hfmm_matvec_df needs a plan created with precision = 1";
        return HFMM_E_INVALID;
    }
    HFMM_GUARD_BEGIN
    run_matvec_df(P, (const float4*)density_df, (float4*)potential_df, parts, (cudaStream_t)stream);
    return HFMM_OK;
    HFMM_GUARD_END
}

int hfmm_matvec(hfmm_plan* P, const void* density, void* potential, int nrhs, void* stream) {
    return hfmm_matvec_parts(P, density, potential, nrhs, 7, stream);
}

int hfmm_matvec_host(hfmm_plan* P, const void* density, void* potential, int nrhs, void* stream) {
    if (!P || !density || !potential || nrhs < 1) return HFMM_E_INVALID;
    HFMM_GUARD_BEGIN
    cudaStream_t st = (cudaStream_t)stream;
    const int R = std::min(nrhs, 64);
    const size_t need = (size_t)R * (size_t)P->N;
    if (P->hio_in.n < need) {
        P->hio_in.alloc(need, &P->dev_bytes);
        P->hio_out.alloc(need, &P->dev_bytes);
    }
    for (int r0 = 0; r0 < nrhs; r0 += R) {
        const int Rc = std::min(R, nrhs - r0);
        const size_t off = (size_t)r0 * (size_t)P->N, bytes = sizeof(float2) * (size_t)Rc * (size_t)P->N;
        HFMM_CUDA(cudaMemcpyAsync(P->hio_in.p, (const float2*)density + off, bytes, cudaMemcpyHostToDevice, st));
        const int s = hfmm_matvec_parts(P, P->hio_in.p, P->hio_out.p, Rc, 7, stream);
        if (s != HFMM_OK) return s;
        HFMM_CUDA(cudaMemcpyAsync((float2*)potential + off, P->hio_out.p, bytes, cudaMemcpyDeviceToHost, st));
    }
    HFMM_CUDA(cudaStreamSynchronize(st));
    return HFMM_OK;
    HFMM_GUARD_END
}

int hfmm_matvec_timed(hfmm_plan* P, const void* density, void* potential, float* stage_ms, void* stream) {
    if (!P || !density || !potential || !stage_ms) return HFMM_E_INVALID;
    cudaEvent_t ev[HFMM_NUM_STAGES + 1] = {};
    HFMM_GUARD_BEGIN
    cudaStream_t st = (cudaStream_t)stream;
    struct Cleanup {
        hfmm_plan* P;
        cudaEvent_t* ev;
        ~Cleanup() {
            P->stage_ev = nullptr;
            for (int q = 0; q <= HFMM_NUM_STAGES; ++q)
                if (ev[q]) cudaEventDestroy(ev[q]);
        }
    } cleanup{P, ev};
    for (int q = 0; q <= HFMM_NUM_STAGES; ++q) HFMM_CUDA(cudaEventCreate(&ev[q]));
    P->stage_ev = ev;
    mark_stage(P, 0, st);
    launch_density_prep(P, density, VecKind::Complex64, P->sig.p, st);
    run_matvec_sorted(P, 7, st);
    launch_output(P, P->phi.p, potential, VecKind::Complex64, st);
    mark_stage(P, HFMM_NUM_STAGES, st);
    HFMM_CUDA(cudaEventSynchronize(ev[HFMM_NUM_STAGES]));
    for (int q = 0; q < HFMM_NUM_STAGES; ++q) HFMM_CUDA(cudaEventElapsedTime(&stage_ms[q], ev[q], ev[q + 1]));
    return HFMM_OK;
    HFMM_GUARD_END
}

int64_t hfmm_launch_count(const hfmm_plan* P) { return P ? P->launches : -1; }

int hfmm_tune_choose(int tunable, const float* ms, int n, int* value) {
    if (tunable < 0 || tunable >= HFMM_NUM_TUNABLES || !ms || !value || n < 1 || n > kTuneCount[tunable])
        return HFMM_E_INVALID;
    int best = -1, def = -1;
    for (int c = 0; c < n; ++c) {
        if (!(ms[c] >= 0.f) || !std::isfinite(ms[c])) continue;  // not measured
        if (best < 0 || ms[c] < ms[best]) best = c;
        if (kTuneValue[tunable][c] == kTuneDefault[tunable]) def = c;
    }
    if (best < 0) return HFMM_E_INVALID;
    // the default stays unless another candidate is at least 2 % faster (timing noise)
    if (def >= 0 && ms[best] > 0.98f * ms[def]) best = def;
    *value = kTuneValue[tunable][best];
    return HFMM_OK;
}

int hfmm_plan_tuning(const hfmm_plan* P, int* choices, float* tuned_ms) {
    if (!P || !choices) return HFMM_E_INVALID;
    choices[0] = P->p2p_variant;
    choices[1] = (P->m2l_variant == 1 && P->n_ts_tiles > 0) ? 1 : 0;
    choices[2] = P->tc_group_used;
    choices[3] = P->mv_mode;
    if (tuned_ms)
        for (int a = 0; a < HFMM_NUM_TUNABLES; ++a)
            for (int c = 0; c < HFMM_TUNE_CANDIDATES; ++c) tuned_ms[a * HFMM_TUNE_CANDIDATES + c] = P->tune_ms[a][c];
    return HFMM_OK;
}

int hfmm_device_status(hfmm_plan* P, void* stream) {
    if (!P) return HFMM_E_INVALID;
    HFMM_GUARD_BEGIN
    cudaStream_t st = (cudaStream_t)stream;
    int flag = 0;
    HFMM_CUDA(cudaMemcpyAsync(&flag, P->dev_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HFMM_CUDA(cudaMemsetAsync(P->dev_err.p, 0, sizeof(int), st));
    HFMM_CUDA(cudaStreamSynchronize(st));
    if (flag) {
        g_last_error = "a device wait gave up (tensor-core M2L)";
        return HFMM_E_TIMEOUT;
    }
    return HFMM_OK;
    HFMM_GUARD_END
}

int hfmm_plan_costs(const hfmm_plan* P, double* costs) {
    if (!P || !costs) return HFMM_E_INVALID;
    for (int q = 0; q < HFMM_NUM_COSTS; ++q) costs[q] = P->cost[q];
    return HFMM_OK;
}

int hfmm_direct(hfmm_plan* P, const void* density, void* potential, int nrhs, void* stream) {
    if (!P || !density || !potential || nrhs < 1) return HFMM_E_INVALID;
    HFMM_GUARD_BEGIN
    cudaStream_t st = (cudaStream_t)stream;
    for (int r = 0; r < nrhs; ++r) {
        launch_density_prep(P, (const float2*)density + (int64_t)r * P->N, VecKind::Complex64, P->sig.p, st);
        run_direct_sorted(P, st);
        launch_output(P, P->phi.p, (float2*)potential + (int64_t)r * P->N, VecKind::Complex64, st);
    }
    HFMM_CUDA(cudaGetLastError());
    return HFMM_OK;
    HFMM_GUARD_END
}

int hfmm_rhs_planewave(hfmm_plan* P, const double* dirs, int nrhs, void* rhs_out, void* stream) {
    if (!P || !dirs || !rhs_out || nrhs < 1) return HFMM_E_INVALID;
    for (int r = 0; r < nrhs; ++r)
        for (int d = 0; d < 3; ++d)
            if (!std::isfinite(dirs[3 * r + d])) return HFMM_E_INVALID;
    HFMM_GUARD_BEGIN
    cudaStream_t st = (cudaStream_t)stream;
    for (int r = 0; r < nrhs; ++r)
        launch_planewave(P, dirs[3 * r], dirs[3 * r + 1], dirs[3 * r + 2], (float2*)rhs_out + (int64_t)r * P->N, st);
    HFMM_CUDA(cudaGetLastError());
    return HFMM_OK;
    HFMM_GUARD_END
}

int hfmm_field(hfmm_plan* P, const void* density, const double* targets, int64_t n_targets, void* field_out,
               void* stream) {
    if (!P || !density || (n_targets > 0 && (!targets || !field_out)) || n_targets < 0) return HFMM_E_INVALID;
    for (int64_t t = 0; t < 3 * n_targets; ++t)
        if (!std::isfinite(targets[t])) return HFMM_E_INVALID;
    HFMM_GUARD_BEGIN
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> tg(targets, targets + 3 * n_targets);
    DBuf<double> d_tg;
    d_tg.upload(tg, nullptr, st);
    run_field(P, (const float2*)density, d_tg.p, n_targets, (float2*)field_out, st);
    HFMM_CUDA(cudaStreamSynchronize(st));  // the target buffer is freed on return
    return HFMM_OK;
    HFMM_GUARD_END
}

int hfmm_solve_refined(hfmm_plan* inner, hfmm_plan* outer, const void* rhs, void* x_out, double tol_outer,
                       int max_outer, int* outer_iters, int* inner_iters, double* relres_out, void* stream) {
    if (!inner || !outer || !rhs || !x_out || !(tol_outer > 0.0) || max_outer < 1) return HFMM_E_INVALID;
    if (inner->N != outer->N || inner->k != outer->k) {
        hfmm_set_last_error("hfmm_solve_refined: the inner and outer plans differ in N or k");
        return HFMM_E_INVALID;
    }
    HFMM_GUARD_BEGIN
    return run_refinement(inner, outer, (const float2*)rhs, (float2*)x_out, tol_outer, max_outer, outer_iters,
                          inner_iters, relres_out, (cudaStream_t)stream);
    HFMM_GUARD_END
}

int hfmm_solve(hfmm_plan* P, const void* rhs, void* x_out, int nrhs, int* iters_out, double* relres_out,
               void* stream) {
    if (!P || !rhs || !x_out || nrhs < 1) return HFMM_E_INVALID;
    HFMM_GUARD_BEGIN
    cudaStream_t st = (cudaStream_t)stream;
    int status = HFMM_OK;
    for (int r0 = 0; r0 < nrhs;) {
        const int R = std::min(nrhs - r0, 64);
        const float2* b = (const float2*)rhs + (int64_t)r0 * P->N;
        float2* x = (float2*)x_out + (int64_t)r0 * P->N;
        if (R > 1 && batch_supported(P, R)) {  // R solves in lockstep on batched matvecs
            std::vector<int> it(R, 0);
            std::vector<double> rr(R, 0.0);
            const int s = run_gmres_batched(P, b, x, R, it.data(), rr.data(), st);
            if (s != HFMM_OK) status = s;
            for (int q = 0; q < R; ++q) {
                if (iters_out) iters_out[r0 + q] = it[q];
                if (relres_out) relres_out[r0 + q] = rr[q];
            }
            r0 += R;
            continue;
        }
        int it = 0;
        double rr = 0.0;
        const int s = run_gmres(P, b, x, &it, &rr, st);
        if (s != HFMM_OK) status = s;
        if (iters_out) iters_out[r0] = it;
        if (relres_out) relres_out[r0] = rr;
        ++r0;
    }
    return status;
    HFMM_GUARD_END
}

}  // extern "C"
