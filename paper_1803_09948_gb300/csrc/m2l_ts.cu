// Target-stationary M2L on the fifth-generation tensor cores (tcgen05, BF16x3).
//
// One block owns a tile of up to 256 consecutive target boxes of one level and keeps
// their local expansions in shared memory (FP32) while it applies every translation
// into them; each local is written to global memory once.  This replaces the
// source-stationary kernel's per-translation bulk reductions into L2, whose per-operation
// cost bounded it.
//
// Operators are shared through the reflection symmetry of the M2L offsets (Sec. 2.3's
// interaction list in a uniform octree: 316 offsets d = c_source - c_target in [-3,3]^3
// with some |d_i| >= 2).  Reflecting the configuration in coordinate planes maps the
// basis functions b_{n,m} = (radial) Q_n^|m|(cos t) e^{i m phi} to signed basis functions
// of the same degree (x -> -x: (-1)^m b_{n,-m}; y -> -y: b_{n,-m}; z -> -z:
// (-1)^{n+m} b_{n,m}), so for a composition R of flips
//     T(R d)[c][c'] = s(c) s(c') T(d)[mu(c)][mu(c')],
// s the product of the signs and mu(m) = -m when exactly one of the x, y flips is
// present (mu is an involution and s(mu(c)) = s(c)).  Hence, with d the canonical offset
// (non-negative components, 56 of them):
//     L_t += T(R d) M_s   <=>   X = S Mu M_s,  y = T(d) X,  L_t += S Mu y,
// a signed permutation of the gathered multipole (done while it is split into BF16 in
// shared memory) and of the product's rows (done while it is added into the tile).
// All translations of a tile that share a canonical operator form one group; the
// operator is loaded once per group into tensor memory (double-buffered), and the group's
// columns (source box, target slot, reflection) go through the MMA in chunks of 64.
//
// Real form and split as in the source-stationary kernel: A rows 2i / 2i+1 are
// [Re T_i, Im T_i] / [Im T_i, -Re T_i] (output coefficient i), B = [Re X; -Im X] with the
// imaginary block at K offset KH = P rounded up to even; A and B are split into BF16
// hi + lo and D = A_hi B_hi + A_hi B_lo + A_lo B_hi accumulates in FP32 in tensor memory.
//
// Roles: warps 0-3 drain the accumulators into the tile (shared-memory atomics through
// the row map), warps 4-11 gather and split B, warp 12 allocates tensor memory and issues
// the MMAs, warps 13-16 load the canonical operators into tensor memory.  Every mbarrier
// wait is bounded; a timeout raises the block's abort flag and the device error flag.
#include <cuda_bf16.h>

#include "hfmm_internal.cuh"
#include "tc_common.cuh"

namespace hfmm {

namespace {

using namespace tc;

constexpr int kM = 128;                          // rows of A / D (2P <= 128)
constexpr int kK = 128;                          // K capacity (2 KH <= 128)
constexpr int kN = 64;                           // columns per chunk
constexpr int kKc = kK / 8;                      // core matrices along K
constexpr uint32_t kCoreBytes = 128;             // 8 rows x 16 bytes
constexpr uint32_t kSBO = kKc * kCoreBytes;      // next 8-row group
constexpr uint32_t kLBO = kCoreBytes;            // next 8-element K group
constexpr int kBElems = kN * kK;                 // BF16 elements per B part
constexpr int kStages = 2;                       // B stages / accumulators in flight
constexpr int kEpi = 128;                        // epilogue threads (warps 0-3)
constexpr int kProd = 256;                       // producer threads (warps 4-11)
constexpr int kMmaWarp = 12;
constexpr int kLoadWarp0 = 13;                   // operator loaders: warps 13-16
constexpr int kMetaWarp = 17;                    // column-list prefetch (bulk copies into a ring)
constexpr int kThreads = 18 * 32;
constexpr int kRing = 8;                         // chunks of column entries in flight
constexpr uint32_t kTmemCols = 512;              // 2 operator buffers (128 each) + 2 accumulators (64 each)
constexpr uint32_t kTmemAcc = 256;
constexpr uint32_t kIdescN64 = idesc_bf16(kM, kN);

// element (r, k) of a K-major core-matrix tile with kKc core matrices per 8-row group
__device__ __forceinline__ uint32_t core_index(uint32_t r, uint32_t k) {
    return ((r >> 3) * kKc + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

struct TsShared {
    __nv_bfloat16 b[kStages][2][kBElems];  // gathered, transformed multipoles: hi, lo per stage
    uint64_t bfull[kStages], bempty[kStages];
    uint64_t afull[kStages], aempty[kStages];
    uint64_t ofull[2], oempty[2];
    uint64_t mfull[kRing], mempty[kRing];  // column-entry ring: bulk copy landed / epilogue done
    alignas(16) int2 ring[kRing][kN];      // column entries of chunks w % kRing (bulk-copy targets)
    int16_t cmap[8][kM / 2];   // [reflection][coefficient q]: mu(q) | 0x4000 when s(q) = -1
    uint32_t tmem;
    int abort;
    // the tile's chunk records (nchunk TsChunk) and then its locals (ntgt x 2P floats) follow
};

__host__ __device__ constexpr size_t ts_fixed_bytes() { return (sizeof(TsShared) + 127) & ~(size_t)127; }

// mu and s of reflection code rc (bit 0 flip x, bit 1 flip y, bit 2 flip z) on coefficient q
__device__ __forceinline__ int16_t refl_entry(int rc, int q) {
    int n = (int)sqrtf((float)q);
    while (n * n > q) --n;
    while ((n + 1) * (n + 1) <= q) ++n;
    const int m = q - n * n - n;
    const bool fx = rc & 1, fy = (rc >> 1) & 1, fz = (rc >> 2) & 1;
    bool neg = false;
    if (fx && (m & 1)) neg = !neg;
    if (fz && ((n + m) & 1)) neg = !neg;
    const int m2 = (fx != fy) ? -m : m;
    return (int16_t)((n * n + n + m2) | (neg ? 0x4000 : 0));
}

// Row r of the real-form operator (r = 2i + part) as BF16 hi/lo pairs into tensor-memory
// columns [base, base + 64) (hi) and [base + 64, base + 128) (lo) of this thread's lane.
// Element k: k < KH -> (part 0: Re T[i][k], part 1: Im T[i][k]) for k < P;
//            k >= KH -> (part 0: Im T[i][k-KH], part 1: -Re T[i][k-KH]) for k - KH < P; else 0.
__device__ __forceinline__ void load_operator_row(const float2* __restrict__ T, int P, int KH, int r,
                                                  uint32_t lane_base, uint32_t base) {
    const int i = r >> 1;
    const bool part = r & 1;
    const bool row_ok = i < P;
    if (P == 64) {
        // two blocks of 32 entries: k = e..e+31 and KH + e..KH + e + 31 are aligned column groups
#pragma unroll 1
        for (int e = 0; e < 64; e += 32) {
            float2 t[32];
            const float4* src = reinterpret_cast<const float4*>(T + (size_t)i * P + e);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float4 v = row_ok ? __ldg(src + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                t[2 * q] = make_float2(v.x, v.y);
                t[2 * q + 1] = make_float2(v.z, v.w);
            }
            uint32_t h1[16], l1[16], h2[16], l2[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float2 a = t[2 * q], b = t[2 * q + 1];
                if (!part) {
                    split_bf16x2(a.x, b.x, h1[q], l1[q]);
                    split_bf16x2(a.y, b.y, h2[q], l2[q]);
                } else {
                    split_bf16x2(a.y, b.y, h1[q], l1[q]);
                    split_bf16x2(-a.x, -b.x, h2[q], l2[q]);
                }
            }
            tmem_st16(lane_base + base + (uint32_t)(e / 2), h1);
            tmem_st16(lane_base + base + 64u + (uint32_t)(e / 2), l1);
            tmem_st16(lane_base + base + (uint32_t)((64 + e) / 2), h2);
            tmem_st16(lane_base + base + 64u + (uint32_t)((64 + e) / 2), l2);
        }
        return;
    }
    // any other order: element by element (plan-size cases only)
#pragma unroll 1
    for (int g = 0; g < 4; ++g) {
        uint32_t h[16], l[16];
#pragma unroll 1
        for (int q = 0; q < 16; ++q) {
            float v2[2];
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int k = 32 * g + 2 * q + h2;
                float v = 0.f;
                if (row_ok) {
                    if (k < KH) {
                        if (k < P) {
                            const float2 tv = __ldg(T + (size_t)i * P + k);
                            v = part ? tv.y : tv.x;
                        }
                    } else if (k - KH < P) {
                        const float2 tv = __ldg(T + (size_t)i * P + (k - KH));
                        v = part ? -tv.x : tv.y;
                    }
                }
                v2[h2] = v;
            }
            split_bf16x2(v2[0], v2[1], h[q], l[q]);
        }
        tmem_st16(lane_base + base + (uint32_t)(16 * g), h);
        tmem_st16(lane_base + base + 64u + (uint32_t)(16 * g), l);
    }
}

__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

__host__ __device__ constexpr size_t ts_chunk_bytes(int max_chunks) {
    return ((size_t)max_chunks * sizeof(TsChunk) + 127) & ~(size_t)127;
}

__global__ void __launch_bounds__(kThreads, 1)
    k_m2l_ts(const TsTile* __restrict__ tiles, const TsChunk* __restrict__ chunks, const int2* __restrict__ cols,
             const float2* __restrict__ canon, float2* __restrict__ coef, int* __restrict__ err, int max_chunks) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TsShared& S = *reinterpret_cast<TsShared*>(smem_raw);
    TsChunk* ch = reinterpret_cast<TsChunk*>(smem_raw + ts_fixed_bytes());  // the tile's chunk records
    float* loc = reinterpret_cast<float*>(smem_raw + ts_fixed_bytes() + ts_chunk_bytes(max_chunks));  // [ntgt][2P]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const TsTile tile = tiles[blockIdx.x];
    const int P = tile.P, KH = (P + 1) & ~1, R2 = 2 * P;
    const int nch = tile.nchunk;
    volatile int* abort = &S.abort;

    if (warp == kMmaWarp) tmem_alloc(smem_u32(&S.tmem), kTmemCols);
    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) {
            mbar_init(smem_u32(&S.bfull[q]), kProd);
            mbar_init(smem_u32(&S.bempty[q]), 1);
            mbar_init(smem_u32(&S.afull[q]), 1);
            mbar_init(smem_u32(&S.aempty[q]), kEpi);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(smem_u32(&S.ofull[q]), 128);
            mbar_init(smem_u32(&S.oempty[q]), 1);
        }
        for (int q = 0; q < kRing; ++q) {
            mbar_init(smem_u32(&S.mfull[q]), 1);
            mbar_init(smem_u32(&S.mempty[q]), kEpi);
        }
        S.abort = 0;
    }
    for (int q = tid; q < nch; q += kThreads) ch[q] = chunks[tile.chunk0 + q];  // one coalesced pass
    for (int e = tid; e < 8 * (kM / 2); e += kThreads) S.cmap[e / (kM / 2)][e % (kM / 2)] = refl_entry(e / (kM / 2), e % (kM / 2));
    for (int e = tid; e < tile.ntgt * R2; e += kThreads) loc[e] = 0.f;
    if (2 * KH < kK) {
        // K rows beyond the real form stay zero in B (A is zero there too), so no stale NaN enters a product
        uint4* bz = reinterpret_cast<uint4*>(&S.b[0][0][0]);
        for (int q = tid; q < (int)(sizeof(S.b) / 16); q += kThreads) bz[q] = make_uint4(0, 0, 0, 0);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;

    if (warp >= 4 && warp < kMmaWarp) {
        // ---------------------------------------------------------------- producers
        const int pt = tid - kEpi;
        for (int w = 0; w < nch; ++w) {
            const int s = w & 1;
            const uint32_t ph = (uint32_t)(w >> 1) & 1u;
            if (!warp_wait(smem_u32(&S.bempty[s]), ph ^ 1u, abort, err)) break;
            const TsChunk c = ch[w];
            const int slot = w % kRing;
            if (!warp_wait(smem_u32(&S.mfull[slot]), (uint32_t)(w / kRing) & 1u, abort, err)) break;
            const int2* ent = S.ring[slot];
            __nv_bfloat16* bh = &S.b[s][0][0];
            __nv_bfloat16* bl = &S.b[s][1][0];
            if (P == 64) {
                // warp q takes columns 8q..8q+7, four lanes per column; lane j the destination
                // coefficient pairs (2(j + 4t), 2(j + 4t) + 1): the 32 lanes' 4-byte stores of one t
                // fill one 128-byte core matrix
                const int cc = (warp - 4) * 8 + (lane >> 2), j = lane & 3;
                if (cc < c.ncol) {
                    const int2 e = ent[cc];
                    const int rc = (e.y >> 16) & 7;
                    const float2* M = coef + tile.src + (int64_t)e.x * 64;
                    float2 a[8], b[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const int q0 = 2 * (j + 4 * t);
                        const int m0 = S.cmap[rc][q0], m1 = S.cmap[rc][q0 + 1];
                        a[t] = __ldg(M + (m0 & 0x3fff));
                        b[t] = __ldg(M + (m1 & 0x3fff));
                        if (m0 & 0x4000) a[t] = make_float2(-a[t].x, -a[t].y);
                        if (m1 & 0x4000) b[t] = make_float2(-b[t].x, -b[t].y);
                    }
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const int q0 = 2 * (j + 4 * t);
                        uint32_t hr, lr, hi, li;
                        split_bf16x2(a[t].x, b[t].x, hr, lr);
                        split_bf16x2(-a[t].y, -b[t].y, hi, li);
                        const uint32_t o_re = core_index(cc, q0), o_im = core_index(cc, 64 + q0);
                        *reinterpret_cast<uint32_t*>(bh + o_re) = hr;
                        *reinterpret_cast<uint32_t*>(bl + o_re) = lr;
                        *reinterpret_cast<uint32_t*>(bh + o_im) = hi;
                        *reinterpret_cast<uint32_t*>(bl + o_im) = li;
                    }
                }
                // columns beyond ncol keep earlier (finite) values: their D columns are never read
            } else {
                for (int task = pt; task < kN * P; task += kProd) {
                    const int cc = task / P, q = task % P;
                    if (cc >= c.ncol) continue;
                    const int2 e = ent[cc];
                    const int m = S.cmap[(e.y >> 16) & 7][q];
                    float2 v = __ldg(coef + tile.src + (int64_t)e.x * P + (m & 0x3fff));
                    if (m & 0x4000) v = make_float2(-v.x, -v.y);
                    __nv_bfloat16 h, l;
                    split_bf16(v.x, h, l);
                    bh[core_index(cc, q)] = h;
                    bl[core_index(cc, q)] = l;
                    split_bf16(-v.y, h, l);
                    bh[core_index(cc, KH + q)] = h;
                    bl[core_index(cc, KH + q)] = l;
                }
            }
            fence_async_smem();  // this thread's stores -> visible to the tensor core
            mbar_arrive(smem_u32(&S.bfull[s]));
        }
    } else if (warp == kMmaWarp) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            int opk = -1, issued = -1;
            const int ksteps = (2 * KH + 15) / 16;
            for (int w = 0; w < nch; ++w) {
                const TsChunk c = ch[w];
                if (c.newop) {
                    ++opk;
                    if (!wait_or_abort(smem_u32(&S.ofull[opk & 1]), (uint32_t)(opk >> 1) & 1u, abort, err)) break;
                }
                const int s = w & 1;
                const uint32_t ph = (uint32_t)(w >> 1) & 1u;
                if (!wait_or_abort(smem_u32(&S.bfull[s]), ph, abort, err)) break;
                if (!wait_or_abort(smem_u32(&S.aempty[s]), ph ^ 1u, abort, err)) break;
                tc_fence_after();
                const uint32_t d = tmem + kTmemAcc + (uint32_t)(s * kN);
                const uint32_t abase = tmem + (uint32_t)((opk & 1) * 128);
                const uint64_t dbh = umma_desc(smem_u32(&S.b[s][0][0]), kLBO, kSBO);
                const uint64_t dbl = umma_desc(smem_u32(&S.b[s][1][0]), kLBO, kSBO);
                constexpr uint64_t kStep = (2 * kLBO) >> 4;  // 16 K elements = 2 core matrices
                for (int k = 0; k < ksteps; ++k) {
                    const uint64_t ko = (uint64_t)k * kStep;
                    const uint32_t ah = abase + (uint32_t)(8 * k), al = abase + 64u + (uint32_t)(8 * k);
                    mma_bf16_ta(d, ah, dbh + ko, kIdescN64, k > 0);
                    mma_bf16_ta(d, ah, dbl + ko, kIdescN64, 1);
                    mma_bf16_ta(d, al, dbh + ko, kIdescN64, 1);
                }
                tc_commit(smem_u32(&S.bempty[s]));
                tc_commit(smem_u32(&S.afull[s]));
                if (w + 1 == nch || ch[w + 1].newop) tc_commit(smem_u32(&S.oempty[opk & 1]));
                issued = w;
            }
            if (*abort && issued >= 0) {
                // drain this thread's MMAs before the tensor memory is released (bounded)
                const int s = issued & 1;
                const uint32_t ph = (uint32_t)(issued >> 1) & 1u;
                for (long long it = 0; it < kWaitLimit; ++it)
                    if (mbar_try_wait(smem_u32(&S.afull[s]), ph)) break;
            }
        }
        __syncwarp();
    } else if (warp >= kLoadWarp0 && warp < kMetaWarp) {
        // ---------------------------------------------------------------- operator loaders
        const int r = 32 * (warp & 3) + lane;  // the TMEM lane this warp may access
        const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
        int opk = -1;
        for (int w = 0; w < nch; ++w) {
            const TsChunk c = ch[w];
            if (!c.newop) continue;
            ++opk;
            if (opk >= 2) {
                bool ok = true;
                if (lane == 0)
                    ok = wait_or_abort(smem_u32(&S.oempty[opk & 1]), ((uint32_t)(opk >> 1) & 1u) ^ 1u, abort, err);
                if (!__shfl_sync(0xffffffffu, (int)ok, 0)) break;
                tc_fence_after();
            }
            load_operator_row(canon + c.op, P, KH, r, lane_base, (uint32_t)((opk & 1) * 128));
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(smem_u32(&S.ofull[opk & 1]));
        }
    } else if (warp == kMetaWarp) {
        // ---------------------------------------------------------------- column-list prefetch
        // chunk w's entries (an even count, 16-byte aligned in global memory) into ring slot w % kRing
        if (lane == 0) {
            for (int w = 0; w < nch; ++w) {
                const int slot = w % kRing;
                if (w >= kRing &&
                    !wait_or_abort(smem_u32(&S.mempty[slot]), ((uint32_t)(w / kRing) & 1u) ^ 1u, abort, err))
                    break;
                const TsChunk c = ch[w];
                const uint32_t bytes = (uint32_t)(((c.ncol + 1) & ~1) * sizeof(int2));
                mbar_arrive_expect_tx(smem_u32(&S.mfull[slot]), bytes);
                bulk_g2s(smem_u32(&S.ring[slot][0]), cols + c.col0, bytes, smem_u32(&S.mfull[slot]));
            }
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- epilogue (warps 0..3)
        const int r = tid;  // TMEM lane = row of D = 2 i + part
        const int i = r >> 1, part = r & 1;
        const bool row_ok = r < R2;
        // this row's destination under each reflection code: byte rc = 2 mu(i) + part (bits
        // 0-6) | sign (bit 7), so a column needs no shared-memory table lookup
        unsigned long long rowmap = 0;
        if (row_ok)
            for (int rc = 0; rc < 8; ++rc) {
                const int m = S.cmap[rc][i];
                const unsigned long long b = (unsigned)(2 * (m & 0x3fff) + part) | ((m & 0x4000) ? 0x80u : 0u);
                rowmap |= b << (8 * rc);
            }
        for (int w = 0; w < nch; ++w) {
            const int s = w & 1;
            const uint32_t ph = (uint32_t)(w >> 1) & 1u;
            const bool ok = warp_wait(smem_u32(&S.afull[s]), ph, abort, err);
            if (!bar_and(ok, 1, kEpi)) break;
            tc_fence_after();
            const int ncol = ch[w].ncol;
            const int slot = w % kRing;
            // landed before the producers used it; this wait makes the entries visible here
            const bool okm = warp_wait(smem_u32(&S.mfull[slot]), (uint32_t)(w / kRing) & 1u, abort, err);
            if (!bar_and(okm, 1, kEpi)) {
                tc_fence_before();
                mbar_arrive(smem_u32(&S.aempty[s]));
                break;
            }
            const int2* ent = S.ring[slot];
            const uint32_t acc = tmem + kTmemAcc + (uint32_t)(s * kN) + ((uint32_t)(warp * 32) << 16);
            // the accumulator in two halves of 32 columns; it is released after the second load.
            // No target repeats within a chunk and every column's rows are a permutation, so the
            // chunk's additions touch distinct words: plain loads and stores, 16 columns at a time
            // (all loads, then all stores).  Chunks run one after another (the epilogue warps
            // meet at the barriers above before each chunk).
#pragma unroll
            for (int hh = 0; hh < kN; hh += 32) {
                float v[32];
                tmem_ld32(acc + (uint32_t)hh, v);
                if (hh + 32 == kN) {
                    tc_fence_before();
                    mbar_arrive(smem_u32(&S.aempty[s]));
                }
                if (!row_ok) continue;
#pragma unroll
                for (int h = 0; h < 32; h += 16) {
                    uint32_t dst[16];
                    float cur[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int y = ent[hh + h + q].y;
                        const uint32_t b = (uint32_t)(rowmap >> (8 * ((y >> 16) & 7))) & 0xffu;
                        dst[q] = (uint32_t)((y & 0xffff) * R2) + (b & 0x7fu) | ((b & 0x80u) << 24);
                        cur[q] = (hh + h + q < ncol) ? loc[dst[q] & 0x7fffffffu] : 0.f;
                    }
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (hh + h + q < ncol)
                            loc[dst[q] & 0x7fffffffu] = cur[q] + ((dst[q] & 0x80000000u) ? -v[h + q] : v[h + q]);
                }
            }
            mbar_arrive(smem_u32(&S.mempty[slot]));  // the ring slot may be refilled
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // the tile's locals into the expansion array (added: the locals may hold other contributions)
    float* out = reinterpret_cast<float*>(coef + tile.dst);
    const int nf = tile.ntgt * R2;
    const int n4 = nf & ~3;
    for (int e = 4 * tid; e < n4; e += 4 * kThreads) red_add_v4(out + e, loc[e], loc[e + 1], loc[e + 2], loc[e + 3]);
    for (int e = n4 + tid; e < nf; e += kThreads) atomicAdd(out + e, loc[e]);
    if (warp == kMmaWarp) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

size_t m2l_ts_smem(int max_tile_floats, int max_chunks) {
    return ts_fixed_bytes() + ts_chunk_bytes(max_chunks) + sizeof(float) * (size_t)max_tile_floats;
}

void m2l_ts_init() {
    static bool done[64] = {};
    int dev = 0;
    HFMM_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && done[dev]) return;
    int optin = 0;
    HFMM_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    HFMM_CUDA(cudaFuncGetAttributes(&fa, k_m2l_ts));
    HFMM_CUDA(cudaFuncSetAttribute(k_m2l_ts, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
    if (dev >= 0 && dev < 64) done[dev] = true;
}

void m2l_ts_launch(const TsTile* tiles, int64_t ntiles, int max_tile_floats, int max_chunks, const TsChunk* chunks,
                   const int2* cols, const float2* canon, float2* coef, int* err, cudaStream_t st) {
    if (ntiles <= 0) return;
    k_m2l_ts<<<(unsigned)ntiles, kThreads, m2l_ts_smem(max_tile_floats, max_chunks), st>>>(tiles, chunks, cols, canon,
                                                                                         coef, err, max_chunks);
    HFMM_CUDA(cudaGetLastError());
}

}  // namespace hfmm
