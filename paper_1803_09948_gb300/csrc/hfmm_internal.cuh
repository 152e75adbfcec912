// Internal declarations of the GB300 Helmholtz FMM library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hfmm.h"

#define HFMM_MAXLEV 21
#define HFMM_PMAX 40          // largest expansion order a plan accepts
#define HFMM_NEAR_CAP 128     // largest near/self triangle set per target
#define HFMM_TRANS_NB 64      // columns per translation work item
constexpr int kP2PTile = 8;   // targets per near-field warp
constexpr int kP2PSub = 4;    // lanes sharing one target (kP2PTile * kP2PSub == 32)
constexpr int kDefaultP2PKernel = 1;  // near-field kernel when the configuration leaves it open
constexpr int kDefaultOverlap = 0;    // two-branch captured matvec when the configuration leaves it open
constexpr int kDefaultM2LKernel = 0;  // tensor-core M2L kernel when the configuration leaves it open

// ---------------------------------------------------------------- errors
struct HfmmError {
    int code;
    std::string what;
};

#define HFMM_CUDA(call)                                                              \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            throw HfmmError{e_ == cudaErrorMemoryAllocation ? HFMM_E_NOMEM : HFMM_E_CUDA, \
                            std::string(#call) + ": " + cudaGetErrorString(e_)};     \
    } while (0)

// records the message returned by hfmm_last_error on the calling thread
void hfmm_set_last_error(const std::string& msg);

// ---------------------------------------------------------------- device buffers
template <typename T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void alloc(size_t count, size_t* counter) {
        release();
        if (count == 0) count = 1;
        HFMM_CUDA(cudaMalloc((void**)&p, count * sizeof(T)));
        n = count;
        if (counter) *counter += count * sizeof(T);
    }
    void upload(const std::vector<T>& h, size_t* counter, cudaStream_t st) {
        alloc(h.size(), counter);
        if (!h.empty())
            HFMM_CUDA(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    }
};

// ---------------------------------------------------------------- translation work
// One work item: Out[:, dst_c] += T * In[:, src_c] for up to HFMM_TRANS_NB column
// pairs.  T is row-major [Pout][Pin] complex64; column c of a coefficient
// array at base offset b is coef[b + c * P .. b + c * P + P).
struct TransItem {
    int64_t op;    // offset (complex elements) of T in the operator buffer
    int64_t src;   // base offset of the source coefficient array
    int64_t dst;   // base offset of the destination coefficient array
    int32_t cols;  // first entry in the column-pair list
    int16_t ncol;  // number of column pairs (<= HFMM_TRANS_NB)
    int16_t pin, pout;  // Pin = (p_in+1)^2, Pout = (p_out+1)^2
    int16_t atomic;     // 1: accumulate with atomics (destinations shared across items)
    int16_t pad[2];
};

// Target-stationary tensor-core M2L (m2l_ts.cu).  A tile holds up to kTsTile consecutive
// target boxes of one level; its translations are grouped by canonical operator (the
// offsets' reflection classes) into chunks of up to kTsChunkCols columns.
constexpr int kTsTile = 128;
constexpr int kTsChunkCols = 128;
constexpr int kTsRows = 128;           // rows of a local in the kernel's real slot form
constexpr int kTsTrash = kTsTile;      // spare row of a tile: padding columns add into it
struct TsTile {
    int64_t dst;     // coef offset (complex elements) of the tile's first local expansion
    int64_t bx;      // offset (16-byte units) of the level's split multipoles (1 KiB per box)
    int32_t P;       // (p+1)^2 of the level (<= 64)
    int32_t ntgt;    // target boxes in the tile
    int32_t chunk0;  // first chunk
    int32_t nchunk;  // chunks
};
struct TsChunk {
    int64_t op;      // offset (BF16 elements) of the canonical operator in the kernel's packed form
    int32_t col0;    // first column: int2 {source box | rc << 24, target slot * kTsRows | rc << 24}, rc
                     // the reflection code (bit 0 x, 1 y, 2 z flipped)
    int16_t ncol;    // columns, a multiple of 8 in 8..kTsChunkCols (padding columns included)
    int16_t newop;   // 1: first chunk of its operator group
};
// a level whose multipoles the target-stationary kernel reads in split form
struct TsSplitLevel {
    int64_t src;   // coef offset of the level's multipoles
    int64_t bx;    // offset (16-byte units) of its split form
    int32_t P;
    int32_t nbox;
};
constexpr int kTsMaxLevels = 16;
struct TsSplitTable {
    TsSplitLevel lev[kTsMaxLevels];
    int nlev;
};

// A run of SIMT translation items of one column width (64, 16 or 8).
struct SimtRange {
    int64_t begin, end;
    int pout_max, width;
};

// per-level constants the adaptive W-list kernels read on the device
struct AdLevel {
    int64_t mofs, lofs;  // this level's multipoles and locals in coef
    int p;               // order
    float s;             // scale min(1, k a)
};

struct LevelInfo {
    int p = 0, P = 0;       // order and (p+1)^2
    double s = 1.0;         // scale min(1, k a)
    double side = 0.0;      // box side
    int64_t nbox = 0;
    int64_t box0 = 0;       // first box of this level in the all-level box arrays
    int64_t mofs = 0;       // offset of this level's multipoles in coef
    int64_t lofs = 0;       // offset of this level's locals in coef
    int64_t m2l_op = 0;     // offset of 343 M2L operators (316 used) [343][P][P]
    int64_t pc_op = 0;      // offset of 8 L2L operators [8][P][P_parent] (levels >= 3)
    int64_t m2m_op = 0;     // offset of 8 M2M operators [8][P_parent][P] (levels >= 3)
    int64_t canon_op = -1;  // offset of the canonical M2L operators in m2l_canon (tensor-core levels)
};

// State of the batched (multiple right-hand side) matvec for R = 2..64 right-hand sides.
// Expansions are laid out [box][rhs][P], so the R expansions of one box are one
// contiguous block and a translation between two boxes is a work item of R columns
// (column index box * R + r); densities and potentials are [point][rhs].
struct BatchState {
    int R = 0;
    DBuf<float2> sig, phi, coef;     // [N][R], [N][R], [coef_total][R]
    DBuf<TransItem> items;           // one item per translation (R columns)
    DBuf<int4> tc_groups;            // tensor-core groups over `items`
    int64_t n_tc_m2l = 0;            // the first n_tc_m2l groups are M2L
    std::vector<std::pair<int64_t, int64_t>> m2m_tc, l2l_tc;       // group ranges per level
    std::vector<std::pair<int64_t, int64_t>> m2m_items, l2l_items;  // item ranges per level (SIMT)
    std::vector<SimtRange> m2l_simt;
    cudaStream_t cap_stream = nullptr;  // private stream the graph is captured on
    cudaGraphExec_t graph = nullptr;    // the captured batched matvec
    const void* g_in = nullptr;
    void* g_out = nullptr;
    int64_t g_launches = 0;             // kernels in one replay
    ~BatchState() {
        if (graph) cudaGraphExecDestroy(graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
};

// The single right-hand-side matvec (sorted densities -> sorted potentials) captured as a
// CUDA graph: with the near field on a side branch (overlap = 1), or its stages one after
// another (overlap = 0); see run_matvec_sorted.
struct MatvecGraph {
    cudaStream_t cap = nullptr, side = nullptr;  // capture stream and the near-field branch
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaGraphExec_t graph = nullptr;      // two branches
    cudaGraphExec_t seq = nullptr;        // one chain
    int64_t launches = 0, seq_launches = 0;  // kernels in one replay
    void reset() {
        if (graph) cudaGraphExecDestroy(graph);
        if (seq) cudaGraphExecDestroy(seq);
        graph = nullptr;
        seq = nullptr;
    }
    ~MatvecGraph() {
        reset();
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (side) cudaStreamDestroy(side);
        if (cap) cudaStreamDestroy(cap);
    }
};

struct alignas(32) PointW64 {
    double x, y, z, w;
};

struct hfmm_plan {
    hfmm_config cfg;
    double k = 0.0;
    int64_t N = 0, nt = 0;
    int L = 0;
    double D = 0.0, lo[3] = {0, 0, 0};
    double r_near = 0.0, mean_edge = 0.0;
    LevelInfo lev[HFMM_MAXLEV + 1];
    int64_t nleaf = 0, ntiles = 0;
    int64_t corr_nnz = 0, m2l_count = 0;
    size_t dev_bytes = 0;
    bool poly_p2p = true;   // near field fits the polynomial kernel range
    float p2p_shift = 0.f;  // k * half the side of a level-L box (the unit of leaf_ijk)
    int p2p_cap = 0;        // most source points in one leaf's neighbourhood (staged near field)
    int p2p_variant = 0;    // near-field kernel: 0 staged (4 lanes per target), 1 packed FP32x2 pairs

    // sorted point data
    DBuf<float4> pts;        // k * (x - leaf centre), sorted
    DBuf<int32_t> perm;      // sorted -> user
    DBuf<int32_t> iperm;     // user -> sorted
    DBuf<float> wscale;      // k w / (4 pi), sorted
    DBuf<int32_t> pt_leaf;   // leaf of each sorted point
    DBuf<double> x64;        // user-order FP64 points (N x 3)
    std::vector<double> host_x, host_w;  // user-order points and weights (host copies)
    std::vector<int32_t> host_t;         // triangle of each point
    // leaves
    DBuf<int32_t> leaf_start;  // nleaf + 1
    DBuf<int4> leaf_ijk;       // centre in units of half a level-L side: (2 ijk + 1) 2^(L - level)
    bool adaptive = false;     // leaves at several levels (else every leaf is at level L)
    DBuf<int32_t> leaf_lev;    // adaptive: level of each leaf
    DBuf<int32_t> leaf_box;    // adaptive: index of each leaf among its level's boxes
    std::vector<int> leaf_levels;  // levels that hold leaves (ascending)
    // adaptive W lists: for leaf t, entries w_ptr[t] .. w_ptr[t+1] name boxes (centre in half
    // level-L sides and level in w_c2, index among their level's boxes in w_idx) whose
    // multipoles are evaluated at t's points, and which take t's points into their locals
    DBuf<int32_t> w_ptr, w_idx, w_leaf;
    DBuf<int4> w_c2;
    DBuf<AdLevel> ad_lev;
    int64_t n_w = 0;
    int w_maxP = 0;            // largest (p+1)^2 among the W boxes' levels
    int p2p_maxnbr = 27;       // most source leaves in one leaf's near list
    DBuf<int32_t> nbr_ptr, nbr;
    DBuf<int4> tiles;          // (leaf, first point, count, 0)
    // far field
    DBuf<float2> coef;         // all multipoles and locals
    int64_t coef_m_total = 0, coef_total = 0;
    DBuf<float2> ops;          // all translation operators
    DBuf<TransItem> items;
    DBuf<int2> item_cols;
    std::vector<TransItem> host_items;  // host copies, for the batched work lists
    std::vector<int2> host_cols;
    std::vector<int4> host_groups;
    std::vector<int64_t> m2m_items_begin, m2m_items_end;  // per level l (parents at l)
    std::vector<int64_t> l2l_items_begin, l2l_items_end;  // per level l (children at l)
    int64_t m2l_items_begin = 0, m2l_items_end = 0;
    std::vector<SimtRange> m2l_simt;  // M2L item ranges on the SIMT kernel
    DBuf<uint16_t> aops;       // tensor-core M2L operators (BF16 hi/lo, packed)
    DBuf<int4> tc_groups;      // (first item, item count, operator, P) per tensor-core block
    DBuf<uint16_t> m2l_canon;  // canonical M2L operators of the tensor-core levels, packed BF16 (m2l_ts.cu)
    DBuf<TsTile> ts_tiles;     // target-stationary M2L work (m2l_ts.cu)
    DBuf<TsChunk> ts_chunks;
    DBuf<int2> ts_cols;
    DBuf<uint4> ts_bx;         // split multipoles of the tensor-core levels (1 KiB per box)
    TsSplitTable ts_split{};
    int64_t ts_split_boxes = 0;
    int64_t n_ts_tiles = 0;
    int ts_max_chunks = 0;
    int64_t n_tc_groups = 0;   // the first n_tc_groups groups are M2L
    std::vector<std::pair<int64_t, int64_t>> m2m_tc, l2l_tc;  // tensor-core group ranges per level
    DBuf<int> dev_err;         // set by kernels whose bounded waits gave up
    // correction
    DBuf<int64_t> corr_ptr;
    DBuf<int32_t> corr_col;
    DBuf<float2> corr_val;
    DBuf<double2> corr_val64;  // precision = 1: the same values in FP64
    // precision = 1: FP64 near field and correction (accurate.cu)
    DBuf<PointW64> acc_xw;     // sorted FP64 positions and k w / (4 pi)
    DBuf<double2> acc_sig, acc_phi;
    // scratch (one matvec at a time per plan)
    DBuf<float2> sig, phi;
    // device staging of hfmm_matvec_host (allocated on first use, kept)
    DBuf<float2> hio_in, hio_out;
    // GMRES workspace (allocated on first solve, kept resident)
    DBuf<float4> kry;          // (restart + 1) x N, double-float complex
    DBuf<float4> gw, gx, gb;   // work vector, iterate, right-hand side (double-float complex)
    DBuf<double> gred;         // reduction scratch
    int kry_m = 0;
    // batched GMRES workspace: (restart + 1) x R x N basis, work vectors, complex64 staging
    DBuf<float4> bkry, bgw, bgx, bgb;
    DBuf<float2> bin, bout;
    DBuf<double> bred;
    int bkry_m = 0, bkry_R = 0;
    // off-surface evaluation: staged sources (position hi, position lo, strength)
    DBuf<float4> fsrc_hi, fsrc_lo;
    DBuf<double> w_user;
    // refinement workspace: right-hand side, iterate, residual (double-float), FP32 staging
    DBuf<float4> rb, rx, rr;
    DBuf<float2> r32, d32;
    DBuf<double> rred;
    int64_t launches = 0;       // kernels launched by this plan
    double cost[HFMM_NUM_COSTS] = {};  // see hfmm_plan_costs
    cudaEvent_t* stage_ev = nullptr;  // set by hfmm_matvec_timed: events after each stage
    BatchState batch;
    int mv_mode = 1;    // 0: stages launched one after another; 1: two-branch captured graph
    int m2l_variant = 0;   // tensor-core M2L: 0 source-stationary items, 1 target-stationary tiles
    int tc_group_used = 32;
    int64_t tc_m2l_base = 0;  // source-stationary M2L groups as built (at most m2l_tc_max_group() items)
    std::vector<std::pair<int64_t, int64_t>> m2m_tc_base, l2l_tc_base;
    float tune_ms[HFMM_NUM_TUNABLES][HFMM_TUNE_CANDIDATES] = {{-1, -1, -1, -1}, {-1, -1, -1, -1},
                                                             {-1, -1, -1, -1}, {-1, -1, -1, -1}};
    MatvecGraph mvg;
    cudaEvent_t host_ev = nullptr;  // blocking-sync event for the solvers' host waits
    cudaGraphExec_t gm_exec = nullptr;  // a GMRES cycle as one launch (while node over one step)
    int64_t gm_launches = 0;            // kernels in one step
    int gm_used = 0;                    // the last single-RHS solve ran its cycles as graph launches
    ~hfmm_plan() {
        if (gm_exec) cudaGraphExecDestroy(gm_exec);
        if (host_ev) cudaEventDestroy(host_ev);
    }
};

// ---------------------------------------------------------------- kernels: FMM matvec
namespace hfmm {

// *p += v without returning the old value (a reduction, not an atomic exchange)
__device__ __forceinline__ void red_add(float2* p, float2 v) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v.x), "f"(v.y) : "memory");
}

// Complex vectors the matvec reads and writes: complex64, or double-float complex
// (float4 = re_hi, im_hi, re_lo, im_lo; value = hi + lo) for the Krylov solver.
enum class VecKind { Complex64, DoubleFloat };
// sig_sorted = k w / (4 pi) * density[perm]  (one right-hand side)
void launch_density_prep(hfmm_plan* P, const void* density, VecKind kind, float2* sig, cudaStream_t st);
// out[perm[i]] = phi[i]
void launch_output(hfmm_plan* P, const float2* phi, void* out, VecKind kind, cudaStream_t st);
// parts bit 0 near, 1 far, 2 correction; writes P->phi
void run_matvec_sorted(hfmm_plan* P, int parts, cudaStream_t st);
// precision = 1 plans (accurate.cu): FP64 point data at plan creation; the double-float matvec
// (user-order float4 in / out; parts as in hfmm_matvec_parts), FP64 near field and correction
void accurate_setup(hfmm_plan* P, cudaStream_t st);
void run_matvec_df(hfmm_plan* P, const float4* in, float4* out, int parts, cudaStream_t st);
// sets the matvec kernels' shared-memory limits on the current device (once; before any capture)
void matvec_kernels_init();
// records stage event q (if timing is active)
void mark_stage(hfmm_plan* P, int q, cudaStream_t st);
void run_direct_sorted(hfmm_plan* P, cudaStream_t st);
// field at targets (device doubles [n][3]) of the density (device complex64, user order)
void run_field(hfmm_plan* P, const float2* density, const double* targets, int64_t nt, float2* out, cudaStream_t st);
// Batched matvec for R right-hand sides (BatchState): whether this plan supports it,
// building the work lists and buffers, and one matvec (density, potential: device
// complex64, N x R column-major, user order).
bool batch_supported(const hfmm_plan* P, int R);
void batch_setup(hfmm_plan* P, int R, cudaStream_t st);
void run_matvec_batched(hfmm_plan* P, const float2* density, float2* potential, cudaStream_t st);
void launch_planewave(hfmm_plan* P, double dx, double dy, double dz, float2* out, cudaStream_t st);
// copies the normalised Legendre recurrence tables to the current device (once per device)
void upload_legendre_tables();

// ---------------------------------------------------------------- kernels: plan build (FP64)
struct ProjectionJob {
    int type;          // 0: regular functions, 1: outgoing functions
    int pf, pb;        // orders of the functions and of the projection basis
    double sf, sb;     // scales
    double rho;        // projection radius
    int nth, nph;      // quadrature
    int nops;          // number of operators
    const double* d0;  // host: nops x 3 vectors (function centre - sphere centre)
    float2* out;       // device: nops x [Pb][Pf]
    bool conj_transpose_copy;  // also write T^H to out2
    float2* out2;      // device: nops x [Pf][Pb]
};
void build_projection_ops(const ProjectionJob& job, double k, cudaStream_t st);
// out[op] = the operator of offset op from canonical operators by coordinate reflections;
// map[op] = (canonical index, flip x, flip y, flip z) (device)
void expand_m2l_reflections(const float2* canon, int P, int nops, const int4* map, float2* out, cudaStream_t st);

struct CorrInputs {
    const double* x64s;     // sorted FP64 points (N x 3)
    const int32_t* tri_s;   // triangle of each sorted point
    const double* V;        // vertices (device)
    const int32_t* F;       // triangles (device)
    const int32_t* iperm;   // user -> sorted
    const double* w64s;     // sorted FP64 weights
    const uint64_t* skey;   // sorted keys of the search-level boxes
    const int32_t* sstart;  // point ranges of the search-level boxes (nsbox + 1)
    int64_t nsbox;
    int search_level, L;
    const int4* pt_ijk;     // level-L integer coordinates of each sorted point
    int64_t N;
    double k, r_near;
    int quad_order;
};
// Returns nnz; fills P->corr_ptr / corr_col / corr_val.
int64_t build_correction(hfmm_plan* P, const CorrInputs& in, cudaStream_t st);

// ---------------------------------------------------------------- octree on the device
// Morton keys (20 bits per axis) of the user-order points x (N x 3) in the cube
// [lo, lo + 2^20 / scale)^3, sorted stably: keys_sorted[i], perm[i] = user index.
void tree_sort_points(const double* x, int64_t N, const double lo[3], double scale, uint64_t* keys_sorted,
                      int32_t* perm, cudaStream_t st);
struct LeafData {      // per sorted point i
    float4* pts;       // k (x - centre of the point's leaf)
    float* wscale;     // k w / (4 pi)
    int32_t* pt_leaf;  // leaf index
    int4* pt_ijk;      // integer coordinates of the point's cell at the deepest level L
    double* x64s;      // sorted FP64 points (N x 3)
    double* w64s;      // sorted FP64 weights
    int32_t* tri_s;    // triangle of the point
    int32_t* iperm;    // user -> sorted (written at iperm[perm[i]])
};
// keys: the sorted point keys; leaf_c2: each leaf's centre in units of half the side of a
// level-L box ((2 ijk + 1) 2^(L - l) for a leaf at level l), so centre = lo + c2 * half_side
void tree_leaf_data(const double* x, const double* w, const int32_t* tri, const int32_t* perm, const uint64_t* keys,
                    int L, const int4* leaf_c2, const int32_t* leaf_start, int64_t nleaf, int64_t N,
                    const double lo[3], double half_side, double k, const LeafData& out, cudaStream_t st);
// 27-box neighbour lists of the leaves (self included, order dx, dy, dz); also returns
// the host copy of the list offsets and each leaf's neighbourhood point count.
void tree_leaf_neighbours(const uint64_t* leaf_key, const int32_t* leaf_start, int64_t nleaf, int L,
                          DBuf<int32_t>& nbr_ptr, DBuf<int32_t>& nbr, std::vector<int32_t>& h_ptr,
                          std::vector<int64_t>& h_hood, size_t* bytes, cudaStream_t st);
// M2L interaction pairs (source box, target box) of one level with nbox sorted keys,
// bucketed by offset slot (slot[343] maps an offset in [-3,3]^3 to 0..315): bucket g is
// pairs[bstart[g] .. bstart[g+1]), targets ascending.  Returns the pair count.
int64_t tree_m2l_lists(const uint64_t* key, int64_t nbox, int l, const int16_t* slot, std::vector<int2>& pairs,
                       std::vector<int64_t>& bstart, cudaStream_t st);

// ---------------------------------------------------------------- tensor-core M2L
size_t m2l_tc_op_elems();  // BF16 elements per packed operator (hi + lo)
int m2l_tc_max_group();    // work items per tensor-core block
void m2l_tc_pack(const float2* T, int P, int nops, uint16_t* out, cudaStream_t st);
void m2l_tc_init();        // sets the kernel's shared-memory limit on the current device (idempotent)
// rhs > 1: batched items, each holding one (source box, target box) pair in `cols` and
// standing for the rhs columns (box * rhs + r); their src / dst offsets are already scaled
void m2l_tc_launch(const int4* groups, int64_t ngroups, const TransItem* items, const int2* cols,
                   const uint16_t* aops, float2* coef, int* err, int rhs, cudaStream_t st);
// target-stationary M2L: one block per tile; canon holds the canonical FP32 operators
void m2l_ts_init();  // shared-memory limit on the current device (idempotent; before any capture)
size_t m2l_ts_smem(int max_chunks);
// the canonical operators T [nops][P][P] (P <= 64) in the kernel's packed form: per operator the
// real-form A (128 rows, K = 128, BF16 hi then lo) in 16 pieces of 4 KiB (kTsOpElems BF16 each op)
constexpr int64_t kTsOpElems = 128 * 256;
void m2l_ts_pack_ops(const float2* T, int P, int nops, uint16_t* out, cudaStream_t st);
// the levels' multipoles in the kernel's split form (BF16 hi / lo of Re and -Im in slot order,
// plain and with the orders reversed), `boxes` boxes in all
void m2l_ts_split(const TsSplitTable& t, int64_t boxes, const float2* coef, uint4* bx, cudaStream_t st);
void m2l_ts_launch(const TsTile* tiles, int64_t ntiles, int max_chunks, const TsChunk* chunks, const int2* cols,
                   const uint16_t* canon, const uint4* bx, float2* coef, int* err, cudaStream_t st);

// ---------------------------------------------------------------- GMRES
int run_gmres(hfmm_plan* P, const void* rhs, void* x, int* iters, double* relres, cudaStream_t st);
// G single right-hand-side solves on distinct plans, cycles of all of them in one graph launch
int run_gmres_group(hfmm_plan* const* plans, int G, const void* const* rhs, void* const* x_out, int* iters,
                    double* relres, cudaStream_t st);
// R (2..64) systems with the same operator in lockstep: one batched matvec per iteration,
// an independent Arnoldi process per right-hand side. rhs, x: device complex64 [R][N].
int run_gmres_batched(hfmm_plan* P, const float2* rhs, float2* x, int R, int* iters, double* relres,
                      cudaStream_t st);
int run_refinement(hfmm_plan* inner, hfmm_plan* outer, const float2* rhs, float2* x, double tol, int max_outer,
                   int* outer_iters, int* inner_iters, double* relres, cudaStream_t st);
// the batched matvec through the plan's captured graph (density, potential: complex64 [R][N])
void batched_matvec(hfmm_plan* P, const float2* d, float2* o, int R, cudaStream_t st);

// host special functions (plan building only)
void host_jn_scaled(int nmax, double z, double s, double* out);
void host_hn_scaled(int nmax, double z, double s, double* re, double* im);

}  // namespace hfmm
