// M2L on the fifth-generation tensor cores (tcgen05, TMEM accumulators), BF16x3.
//
// One work item applies the translation matrix T of one offset (Sec. 2.3's M2L,
// Eq. 11-14 read as the local/multipole addition theorem) to up to 64 gathered
// multipole columns X and accumulates into the targets' local expansions:
//     L[:, dst_c] += T X[:, src_c].
// In real arithmetic with interleaved rows
//     A = rows 2i: [Re T_i, Im T_i],  rows 2i+1: [Im T_i, -Re T_i]   (128 x 2P)
//     B = [Re X ; -Im X]                                           (2P x 64)
//     D = A B:  row 2i = Re (T X)_i,  row 2i+1 = Im (T X)_i.
// A and B are split into BF16 high and low parts (x = hi + lo, 16 significant
// bits), and D = A_hi B_hi + A_hi B_lo + A_lo B_hi is accumulated in FP32 in
// tensor memory: tcgen05.mma kind::f16, M = 128, N = 64 kPair, K = 16 per
// instruction.  A is split once at plan time and, for the work items of one
// offset grouped in a block, held in tensor memory (written once with
// tcgen05.st); B is gathered from the multipole array, split on the fly and
// staged in shared memory in the K-major no-swizzle (core-matrix) layout,
// item kPair m + h in rows 64h..64h+63 of step m's stage.
//
// Roles per block: producer warps gather and split B; one thread issues the
// MMAs; four epilogue warps move each accumulator from tensor memory into one
// of several shared-memory output stages; two issuer warps add the staged
// expansions into global memory with bulk-copy reductions (a run of
// consecutive destination boxes is one contiguous reduction).  The issuers are
// decoupled from the epilogue so that the bulk-copy engine, whose per-operation
// cost bounds the output, stays busy while the next accumulator drains.
//
// The output path bounds the kernel: with two issuers, four output stages of
// one item each run 0.75 ms on the 1.97 M-point workload and three run 1.5 ms
// (the epilogue then waits for every commit); half-item output units (eight
// stages) and two items per N = 128 MMA (which issues in the time of one N = 64
// MMA, half the tensor-pipe cycles per item) both measured slower, so kPair = 1
// and kOutCols = 64.
#include <cuda_bf16.h>

#include "hfmm_internal.cuh"
#include "tc_common.cuh"

namespace hfmm {

namespace {

constexpr int kM = 128;        // rows of A (2P <= 128)
constexpr int kK = 128;        // K (2P rounded up; P <= 64)
constexpr int kN = 64;         // columns per work item
constexpr int kPair = 1;       // work items per MMA step (consecutive items of the group)
constexpr int kNP = kPair * kN;  // columns per MMA
constexpr int kKc = kK / 8;    // core matrices along K
constexpr uint32_t kCoreBytes = 128;                 // 8 rows x 16 bytes
constexpr uint32_t kSBO = kKc * kCoreBytes;          // next 8-row group
constexpr uint32_t kLBO = kCoreBytes;                // next 8-element K group
constexpr uint32_t kTmemCols = kNP;  // one accumulator: kNP FP32 columns
constexpr uint32_t kTmemA = 128;      // A hi (64 columns) and lo (64 columns): 128 x 128 BF16 each

// element (r, k) of a K-major core-matrix tile with kKc core matrices per 8-row group
__host__ __device__ constexpr uint32_t core_index(uint32_t r, uint32_t k) {
    return ((r >> 3) * kKc + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

using namespace tc;

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr) { return tc::umma_desc(addr, kLBO, kSBO); }

// kind::f16 instruction descriptor: D f32, A/B bf16, both K-major, N = kNP, M = 128
constexpr uint32_t kIdesc = idesc_bf16(kM, kNP);

__device__ __forceinline__ void mma_bf16_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t accumulate) {
    tc::mma_bf16_ta(tmem_d, tmem_a, b, kIdesc, accumulate);
}

// Operator conversion (plan time): FP32 complex T [P][P] -> A_hi, A_lo (row-major BF16).
__global__ void k_m2l_tc_pack(const float2* __restrict__ T, int P, int nops, __nv_bfloat16* __restrict__ out) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nops * kM * kK) return;
    int op = (int)(idx / (kM * kK));
    int rk = (int)(idx % (kM * kK));
    int r = rk / kK, k = rk % kK;
    int i = r >> 1;
    bool odd = r & 1;
    float v = 0.f;
    if (i < P) {
        const float2* row = T + (int64_t)op * P * P + (int64_t)i * P;
        if (k < P) v = odd ? row[k].y : row[k].x;
        else if (k < 2 * P) v = odd ? -row[k - P].x : row[k - P].y;
    }
    __nv_bfloat16 hi, lo;
    split_bf16(v, hi, lo);
    __nv_bfloat16* o = out + (int64_t)op * 2 * kM * kK;
    o[r * kK + k] = hi;  // row-major: row r is TMEM lane r, two K elements per column
    o[kM * kK + r * kK + k] = lo;
}

constexpr int kStages = 2;         // B stages and TMEM accumulators in flight (kPair items each)
constexpr int kOutCols = 64;       // columns per output unit (an item holds kN / kOutCols units)
constexpr int kUnits = kN / kOutCols;
constexpr int kCpl = kOutCols / 32;  // unit columns per issuer lane
constexpr int kOutStages = 4;      // shared-memory output stages (epilogue -> issuers), one unit each
constexpr int kIssuers = 2;        // output-issuing warps; issuer q takes units q, q + 2, ...
constexpr int kMaxGroup = 32;      // work items per block (one operator)
constexpr int kProducers = 256;    // threads gathering B (warps 4..11)
constexpr int kEpilogue = 128;     // threads draining TMEM (warps 0..3, one per TMEM lane quarter)
constexpr int kMmaWarp = (kEpilogue + kProducers) / 32;  // TMEM owner and MMA issuer
constexpr int kIssuerWarp = kMmaWarp + 1;                // first output-issuing warp
constexpr int kThreads = kEpilogue + kProducers + 32 + 32 * kIssuers;
// A (128 columns) + kStages accumulators, rounded up to a power of two
constexpr uint32_t kTmemAlloc = kTmemA + kStages * kTmemCols <= 256 ? 256 : 512;
static_assert(kTmemA + kStages * kTmemCols <= kTmemAlloc, "tensor memory budget");
// the epilogue reuses the stage of unit u - kOutStages, which its issuer frees after
// committing its next unit u - kOutStages + kIssuers: that unit must precede u
static_assert(kOutStages > kIssuers, "output stages must outnumber the issuers");
static_assert(kN % kOutCols == 0 && kOutCols % 32 == 0, "output units: whole warps of columns");

struct TcSmem {
    __nv_bfloat16 b[kStages][2][kNP * kK];  // gathered multipoles of kPair items: hi, lo per stage
    float stage[kOutStages][kOutCols][kM];  // accumulator columns = target expansions (Re/Im interleaved)
    uint64_t full[kStages];                 // producers -> MMA: stage written
    uint64_t empty[kStages];                // MMA done reading the stage
    uint64_t tfull[kStages];                // accumulator ready
    uint64_t tempty[kStages];               // epilogue done reading the accumulator
    uint64_t staged[kOutStages];            // epilogue -> issuer: output stage written
    uint64_t sfree[kOutStages];             // issuer -> epilogue: stage read by the bulk engine
    TransItem items[kMaxGroup];             // the group's work items
    uint32_t tmem;
    int abort;
};
static_assert(sizeof(TcSmem) <= 232448, "one block per SM: at most 227 KiB of shared memory");

// AND of v over the 128 epilogue threads (named barrier 1)
__device__ __forceinline__ bool epilogue_all(bool v) { return bar_and(v, 1, 128); }

// Column pair c of a work item: (source, destination) column.  A batched item (rhs > 1)
// is one box pair whose rhs right-hand sides are consecutive columns.
__device__ __forceinline__ int2 item_col(const int2* __restrict__ cols, const TransItem& it, int c, int rhs) {
    if (rhs > 1) {
        const int2 pr = __ldg(cols + it.cols);
        return make_int2(pr.x * rhs + c, pr.y * rhs + c);
    }
    return __ldg(cols + it.cols + c);
}

__global__ void __launch_bounds__(kThreads, 1)
    k_m2l_tc(const int4* __restrict__ groups, const TransItem* __restrict__ items, const int2* __restrict__ cols,
             const __nv_bfloat16* __restrict__ aops, float2* __restrict__ coef, int* __restrict__ err, int rhs) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int4 g = groups[blockIdx.x];  // (first item, item count, operator index, P)
    const int P = g.w, nitems = g.y;
    const int nsteps = (nitems + kPair - 1) / kPair;  // MMA steps: items kPair m .. kPair m + kPair - 1
    volatile int* abort = &S.abort;

    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                     "r"(kTmemAlloc)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) {
            mbar_init(smem_u32(&S.full[q]), kProducers);
            mbar_init(smem_u32(&S.empty[q]), 1);
            mbar_init(smem_u32(&S.tfull[q]), 1);
            mbar_init(smem_u32(&S.tempty[q]), kEpilogue);
        }
        for (int q = 0; q < kOutStages; ++q) {
            mbar_init(smem_u32(&S.staged[q]), kEpilogue);
            mbar_init(smem_u32(&S.sfree[q]), 1);
        }
        S.abort = 0;
    }
    // the operator rows (epilogue warps: thread r holds row r, hi then lo) are requested
    // first, so that their latency overlaps the item-list load below
    uint4 arow[16];
    const uint4* asrc = reinterpret_cast<const uint4*>(aops + (int64_t)g.z * 2 * kM * kK) + (size_t)(tid & 127) * (kK / 8);
    if (warp < 4) {
#pragma unroll
        for (int q = 0; q < 16; ++q) arow[q] = __ldg(asrc + q);
    }
    for (int q = tid; q < nitems; q += kThreads) S.items[q] = items[g.x + q];
    __syncthreads();
    // the group's column lists into L2 (lines of 16 entries, and the last entry of each
    // list), so that the producers' and issuers' per-item reads do not wait on DRAM
    for (int q = tid; q < nitems * 5; q += kThreads) {
        const TransItem& it = S.items[q / 5];
        const int n = rhs > 1 ? 1 : it.ncol;
        const int e = min(16 * (q % 5), n - 1);
        if (e >= 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(cols + it.cols + e));
    }
    if (2 * P < kK) {
        // K beyond 2P stays zero in B (A is zero there too), so no stale NaN enters a product;
        // with 2P = K every element a product reads is written before it is read, and a stale
        // row beyond an item's column count only reaches its own, unused, column of D
        uint4* bz = reinterpret_cast<uint4*>(&S.b[0][0][0]);
        for (int q = tid; q < (int)(sizeof(S.b) / 16); q += kThreads) bz[q] = make_uint4(0, 0, 0, 0);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp < 4) {
        // the group's operator into tensor memory: thread r writes row r (its lane),
        // hi into columns 0..63 and lo into 64..127, two BF16 per column
        const uint32_t lane_base = S.tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int part = 0; part < 2; ++part) {
            if (part == 1) {
#pragma unroll
                for (int q = 0; q < 16; ++q) arow[q] = __ldg(asrc + (kM * kK / 8) + q);
            }
#pragma unroll
            for (int cb = 0; cb < 4; ++cb) {
                uint32_t v[16];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    v[4 * q] = arow[4 * cb + q].x;
                    v[4 * q + 1] = arow[4 * cb + q].y;
                    v[4 * q + 2] = arow[4 * cb + q].z;
                    v[4 * q + 3] = arow[4 * cb + q].w;
                }
                tmem_st16(lane_base + (uint32_t)(part * 64 + cb * 16), v);
            }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;

    if (warp >= 4 && warp < kMmaWarp) {
        // ---------------------------------------------------------------- producers
        // Stage of step m: item kPair m + h in B rows 64h..64h+63.
        const int pt = tid - kEpilogue;
        const int nchunk = (P + 7) >> 3;
        // P = 64: producer warp q takes columns 8q..8q+7 of both items, four lanes per column,
        // each lane the float4s j, j+4, ..., j+28 of its column (complex elements 2(j+4t),
        // 2(j+4t)+1): a load touches 8 lines, and the 32 lanes' 4-byte stores fill one 128-byte
        // core matrix, no bank conflict.  The source columns are read one step ahead and the
        // step's gathers are in flight before the wait for a free stage.
        const bool fast = P == kN && kProducers == 8 * 32;
        const int c = (warp - 4) * 8 + (lane >> 2), j = lane & 3;
        int src[kPair];  // this lane's source column in the next step's items (-1: none)
        auto fetch_src = [&](int m) {
#pragma unroll
            for (int h = 0; h < kPair; ++h) {
                const int w = kPair * m + h;
                src[h] = (w < nitems && c < S.items[w].ncol) ? item_col(cols, S.items[w], c, rhs).x : -1;
            }
        };
        if (fast) fetch_src(0);
        for (int m = 0; m < nsteps; ++m) {
            const int s = m & 1;
            const uint32_t ph = (uint32_t)(m >> 1) & 1u;
            if (fast) {
                int cur[kPair];
#pragma unroll
                for (int h = 0; h < kPair; ++h) cur[h] = src[h];
                if (m + 1 < nsteps) fetch_src(m + 1);
                float4 v[kPair][8];
#pragma unroll
                for (int h = 0; h < kPair; ++h) {
                    const float4* x4 = reinterpret_cast<const float4*>(coef);
                    if (cur[h] >= 0)
                        x4 = reinterpret_cast<const float4*>(coef + S.items[kPair * m + h].src + (int64_t)cur[h] * P);
#pragma unroll
                    for (int t = 0; t < 8; ++t)
                        v[h][t] = cur[h] >= 0 ? __ldg(x4 + j + 4 * t) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                if (!wait_or_abort(smem_u32(&S.empty[s]), ph ^ 1u, abort, err)) break;
#pragma unroll
                for (int h = 0; h < kPair; ++h) {
                    if (cur[h] < 0) continue;
                    __nv_bfloat16* bh = &S.b[s][0][h * kN * kK];
                    __nv_bfloat16* bl = &S.b[s][1][h * kN * kK];
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const float4 x = v[h][t];
                        const __nv_bfloat162 hr = __floats2bfloat162_rn(x.x, x.z);
                        const __nv_bfloat162 hi = __floats2bfloat162_rn(-x.y, -x.w);
                        const float2 br = __bfloat1622float2(hr), bi = __bfloat1622float2(hi);
                        const __nv_bfloat162 lr = __floats2bfloat162_rn(x.x - br.x, x.z - br.y);
                        const __nv_bfloat162 li = __floats2bfloat162_rn(-x.y - bi.x, -x.w - bi.y);
                        const int k = 2 * (j + 4 * t);
                        const uint32_t o_re = core_index(c, k), o_im = core_index(c, P + k);
                        *reinterpret_cast<__nv_bfloat162*>(bh + o_re) = hr;
                        *reinterpret_cast<__nv_bfloat162*>(bl + o_re) = lr;
                        *reinterpret_cast<__nv_bfloat162*>(bh + o_im) = hi;
                        *reinterpret_cast<__nv_bfloat162*>(bl + o_im) = li;
                    }
                }
            } else {
                if (!wait_or_abort(smem_u32(&S.empty[s]), ph ^ 1u, abort, err)) break;
                for (int h = 0; h < kPair && kPair * m + h < nitems; ++h) {
                    const TransItem& it = S.items[kPair * m + h];
                    const int ncol = it.ncol;
                    __nv_bfloat16* bh = &S.b[s][0][h * kN * kK];
                    __nv_bfloat16* bl = &S.b[s][1][h * kN * kK];
                    for (int task = pt; task < kN * nchunk; task += kProducers) {
                        const int cc = task / nchunk, jj = task % nchunk;
                        if (cc >= ncol) continue;
                        const float2* x = coef + it.src + (int64_t)item_col(cols, it, cc, rhs).x * P + 8 * jj;
                        __align__(16) __nv_bfloat16 rh[8], rl[8], ih[8], il[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const float2 v = (8 * jj + q < P) ? __ldg(x + q) : make_float2(0.f, 0.f);
                            split_bf16(v.x, rh[q], rl[q]);
                            split_bf16(-v.y, ih[q], il[q]);
                        }
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            if (8 * jj + q < P) {
                                bh[core_index(cc, 8 * jj + q)] = rh[q];
                                bl[core_index(cc, 8 * jj + q)] = rl[q];
                                bh[core_index(cc, P + 8 * jj + q)] = ih[q];
                                bl[core_index(cc, P + 8 * jj + q)] = il[q];
                            }
                    }
                }
            }
            fence_async_smem();  // this thread's stores -> visible to the tensor core
            mbar_arrive(smem_u32(&S.full[s]));
        }
    } else if (warp == kMmaWarp) {
        // ---------------------------------------------------------------- MMA issuer
        int issued = -1;
        if (lane == 0) {
            for (int m = 0; m < nsteps; ++m) {
                const int s = m & 1;
                const uint32_t ph = (uint32_t)(m >> 1) & 1u;
                if (!wait_or_abort(smem_u32(&S.full[s]), ph, abort, err)) break;
                if (!wait_or_abort(smem_u32(&S.tempty[s]), ph ^ 1u, abort, err)) break;
                tc_fence_after();
                const uint32_t d = tmem + kTmemA + (uint32_t)(s * kTmemCols);
                // B descriptors of K-step 0; a K-step of 16 advances the start address by
                // 2 core matrices, i.e. (2 * kLBO) >> 4 in the descriptor's address field.
                // A of K-step k sits in tensor-memory columns 8k (hi) and 64 + 8k (lo).
                const uint64_t dbh = umma_desc(smem_u32(&S.b[s][0][0])), dbl = umma_desc(smem_u32(&S.b[s][1][0]));
                constexpr uint64_t kStep = (2 * kLBO) >> 4;
#pragma unroll
                for (int k = 0; k < kK / 16; ++k) {
                    const uint64_t ko = (uint64_t)k * kStep;
                    const uint32_t ah = tmem + (uint32_t)(8 * k), al = tmem + 64u + (uint32_t)(8 * k);
                    mma_bf16_ta(d, ah, dbh + ko, k > 0);
                    mma_bf16_ta(d, ah, dbl + ko, 1);
                    mma_bf16_ta(d, al, dbh + ko, 1);
                }
                tc_commit(smem_u32(&S.empty[s]));
                tc_commit(smem_u32(&S.tfull[s]));
                issued = m;
            }
            if (*abort && issued >= 0) {
                // drain this thread's MMAs before the tensor memory is released (bounded)
                const int s = issued & 1;
                const uint32_t ph = (uint32_t)(issued >> 1) & 1u;
                for (long long it = 0; it < kWaitLimit; ++it)
                    if (mbar_try_wait(smem_u32(&S.tfull[s]), ph)) break;
            }
        }
        __syncwarp();
    } else if (warp >= kIssuerWarp) {
        // ---------------------------------------------------------------- output issuers
        // Output unit u is columns [kOutCols h, kOutCols h + kOutCols) of item u / kUnits
        // (h = u % kUnits); lane l handles its unit columns l (and l + 32).  A run of
        // consecutive destination boxes is one contiguous block in both the stage and the
        // expansion array when 2P = kM, and goes out as one reduction; the run starts are a
        // ballot.  Bulk groups are per thread: every lane commits one group per unit and
        // confirms the reads of its previous unit before that unit's stage is handed back.
        const int q = warp - kIssuerWarp;
        // Columns per reduction at most: the bulk engine overlaps several operations, so the
        // contiguous columns of a batched item (one box pair, rhs columns) go out as 2 KiB
        // pieces; single right-hand-side runs are short anyway.
        const int opc = rhs > 1 ? 4 : kN;
        const int nunits = nitems * kUnits;
        int prev = -1;
        if ((P & 1) == 0) {
            // destination columns of this lane's columns, read one unit ahead
            int dn[kCpl];
            auto fetch_dst = [&](int u) {
                const TransItem& it = S.items[u / kUnits];
#pragma unroll
                for (int h = 0; h < kCpl; ++h) {
                    const int c = (u % kUnits) * kOutCols + lane + 32 * h;
                    dn[h] = c < it.ncol ? item_col(cols, it, c, rhs).y : 0;
                }
            };
            if (q < nunits) fetch_dst(q);
            for (int u = q; u < nunits; u += kIssuers) {
                const int o = u % kOutStages;
                const uint32_t po = (uint32_t)(u / kOutStages) & 1u;
                const TransItem& it = S.items[u / kUnits];
                const int cb = (u % kUnits) * kOutCols;  // first item column of the unit
                const int nu = min(it.ncol - cb, kOutCols);  // columns of the unit (may be <= 0)
                int d[kCpl];
#pragma unroll
                for (int h = 0; h < kCpl; ++h) d[h] = dn[h];
                if (u + kIssuers < nunits) fetch_dst(u + kIssuers);
                bool ok = true;
                if (lane == 0) ok = wait_or_abort(smem_u32(&S.staged[o]), po, abort, err);
                if (!__shfl_sync(0xffffffffu, (int)ok, 0)) break;
                bool st[kCpl];
                uint64_t starts = 0;
#pragma unroll
                for (int h = 0; h < kCpl; ++h) {
                    const int j = lane + 32 * h;  // column within the unit
                    st[h] = j < nu;
                    if (2 * P == kM) {
                        // a run starts at the unit's first column, after a break in the
                        // destinations, and every opc item columns
                        const int up = __shfl_up_sync(0xffffffffu, d[h], 1);
                        const int last = __shfl_sync(0xffffffffu, d[h > 0 ? h - 1 : 0], 31);
                        const int pd = lane == 0 ? (h > 0 ? last : d[h] + 1) : up;
                        st[h] = st[h] && (j == 0 || pd != d[h] - 1 || (cb + j) % opc == 0);
                    }
                    starts |= (uint64_t)__ballot_sync(0xffffffffu, st[h]) << (32 * h);
                }
#pragma unroll
                for (int h = 0; h < kCpl; ++h) {
                    if (!st[h]) continue;
                    const int j = lane + 32 * h;
                    uint32_t bytes = 8u * (uint32_t)P;
                    if (2 * P == kM) {
                        // the run ends at the next start, else at the unit's last column
                        const uint64_t later = j < kOutCols - 1 ? starts >> (j + 1) : 0ull;
                        const int end = later ? j + __ffsll((long long)later) : nu;
                        bytes *= (uint32_t)(end - j);
                    }
                    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;" ::"l"(
                                     coef + it.dst + (int64_t)d[h] * P),
                                 "r"(smem_u32(&S.stage[o][j][0])), "r"(bytes)
                                 : "memory");
                }
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                if (prev >= 0) {
                    asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");  // prev's stage read
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&S.sfree[prev % kOutStages]));
                }
                prev = u;
            }
        }
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // every reduction landed
    } else {
        // ---------------------------------------------------------------- epilogue (warps 0..3)
        // The accumulator of step m holds item kPair m + h in columns 64h..64h+63; it is
        // handed back once its last item is in registers.
        const int r = tid;  // TMEM lane = row of D
        const int i = r >> 1;
        const bool odd = r & 1;
        bool stop = false;
        for (int m = 0; m < nsteps && !stop; ++m) {
            const int s = m & 1;
            const uint32_t ph = (uint32_t)(m >> 1) & 1u;
            const bool ok = wait_or_abort(smem_u32(&S.tfull[s]), ph, abort, err);
            if (!epilogue_all(ok)) break;
            tc_fence_after();
            for (int h = 0; h < kPair && kPair * m + h < nitems; ++h) {
                const int w = kPair * m + h;
                const bool last = h == kPair - 1 || w + 1 == nitems;
                const TransItem& it = S.items[w];
                const int ncol = it.ncol;
                const uint32_t base = tmem + kTmemA + (uint32_t)(s * kTmemCols + h * kN) + ((uint32_t)(warp * 32) << 16);
                float v[kN];
                tmem_ld64(base, v);
                if (last) {
                    tc_fence_before();
                    mbar_arrive(smem_u32(&S.tempty[s]));  // accumulator drained: its last item is in v[]
                }
                if ((P & 1) == 0) {
                    // Column c of D, rows 0..2P-1, is the 8P-byte image of the target expansion
                    // L[dst_c] (Re, Im interleaved): stage the columns for the issuer warps, one
                    // output unit of kOutCols columns at a time
#pragma unroll
                    for (int x = 0; x < kUnits; ++x) {
                        const int u = w * kUnits + x;
                        const int o = u % kOutStages;
                        const uint32_t po = (uint32_t)(u / kOutStages) & 1u;
                        const bool fr = wait_or_abort(smem_u32(&S.sfree[o]), po ^ 1u, abort, err);
                        if (!epilogue_all(fr)) {
                            stop = true;
                            break;
                        }
                        if (x * kOutCols < ncol) {
#pragma unroll
                            for (int c = 0; c < kOutCols; ++c) S.stage[o][c][r] = v[x * kOutCols + c];
                            fence_async_smem();
                        }
                        mbar_arrive(smem_u32(&S.staged[o]));
                    }
                    if (stop) break;
                    continue;
                }
                // odd P: per-lane reductions.  Column pairs (c, c+1): the even lane (Re row) sends
                // its c+1 value and takes column c, the odd lane (Im row) the reverse; every lane
                // issues one reduction, no divergent branch
                const bool row_ok = i < P;
#pragma unroll
                for (int c = 0; c < kN; c += 2) {
                    const float send = odd ? v[c] : v[c + 1];
                    const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
                    const int col = c + (odd ? 1 : 0);
                    const float re = odd ? recv : v[c];
                    const float imv = odd ? v[c + 1] : recv;
                    if (row_ok && col < ncol)
                        red_add(coef + it.dst + (int64_t)item_col(cols, it, col, rhs).y * P + i, make_float2(re, imv));
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemAlloc) : "memory");
}

}  // namespace

size_t m2l_tc_op_elems() { return (size_t)2 * kM * kK; }
int m2l_tc_max_group() { return kMaxGroup; }

void m2l_tc_pack(const float2* T, int P, int nops, uint16_t* out, cudaStream_t st) {
    int64_t n = (int64_t)nops * kM * kK;
    k_m2l_tc_pack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(T, P, nops, reinterpret_cast<__nv_bfloat16*>(out));
    HFMM_CUDA(cudaGetLastError());
}

void m2l_tc_init() {
    // once per device, so that a later launch inside a stream capture sets nothing
    static bool attr_set[64] = {};
    int dev = 0;
    HFMM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        HFMM_CUDA(cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcSmem)));
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
}

void m2l_tc_launch(const int4* groups, int64_t ngroups, const TransItem* items, const int2* cols,
                   const uint16_t* aops, float2* coef, int* err, int rhs, cudaStream_t st) {
    if (ngroups <= 0) return;
    const size_t smem = sizeof(TcSmem);
    m2l_tc_init();
    k_m2l_tc<<<(unsigned)ngroups, kThreads, smem, st>>>(groups, items, cols,
                                                   reinterpret_cast<const __nv_bfloat16*>(aops), coef, err, rhs);
    HFMM_CUDA(cudaGetLastError());
}

}  // namespace hfmm
