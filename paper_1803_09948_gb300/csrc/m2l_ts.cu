// Target-stationary M2L on the fifth-generation tensor cores (tcgen05, BF16x3).
//
// One block owns a tile of up to 128 consecutive target boxes of one level and keeps
// their local expansions in shared memory (FP32) while it applies every translation
// into them; each local is written to global memory once.  This replaces the
// source-stationary kernel's per-translation bulk reductions into L2.
//
// Operators are shared through the reflection symmetry of the M2L offsets (Sec. 2.3's
// interaction list in a uniform octree: 316 offsets d = c_source - c_target in [-3,3]^3
// with some |d_i| >= 2).  Reflecting the configuration in coordinate planes maps the
// basis functions b_{n,m} = (radial) Q_n^|m|(cos t) e^{i m phi} to signed basis functions
// of the same degree (x -> -x: (-1)^m b_{n,-m}; y -> -y: b_{n,-m}; z -> -z:
// (-1)^{n+m} b_{n,m}), so for a composition R of flips
//     T(R d)[c][c'] = s(c) s(c') T(d)[mu(c)][mu(c')],
// s the product of the signs and mu(m) = -m when exactly one of the x, y flips is present
// (mu is an involution and s(mu(c)) = s(c)).  With d the canonical offset (non-negative
// components, 56 of them):
//     L_t += T(R d) M_s   <=>   X = S Mu M_s,  y = T(d) X,  L_t += S Mu y.
//
// Coefficient order ("slots").  Expansions of order 7 have 64 coefficients in degree blocks
// of 1, 3, ..., 15.  The kernel orders them so that slots 16g .. 16g+15 hold the whole blocks
// of degrees 7 - g and g (15 - 2g + 2g + 1 = 16), which keeps mu (a reversal inside each
// block) inside one group: on the input side a producer warp owns one group and reverses
// in registers; on the output side the rows of group g are TMEM lanes 32g .. 32g+31, one
// epilogue warp, so the row permutation is one warp shuffle per column.  Lower orders use
// the same 64 slots with the absent degrees empty (zero operator rows and columns).
//
// Real form and split: A rows 2s / 2s+1 are [Re T_s, Im T_s] / [Im T_s, -Re T_s] (output
// slot s, input slots along K), B = [Re X; -Im X] (input slots, K = 128), both split into
// BF16 hi + lo, D = A_hi B_hi + A_hi B_lo + A_lo B_hi accumulated in FP32 in tensor
// memory, M = 128, N = 128 columns per chunk (an N = 128 MMA issues in the time of an
// N = 64 one on this part), K = 16 per instruction.
//
// Source side.  Before the kernel, every source box's multipoles are written once in split
// form: the four rows hi(Re u), hi(-Im u), lo(Re u), lo(-Im u) of 64 BF16 each in slot order,
// once as they are and once with mu applied (1 KiB per box).  A column's B entries are then
// its box's plain or reversed rows with the reflection's signs (sign-bit flips, exact on both
// parts): producer lanes copy 16-byte rows, eight columns per warp instruction, so that a load
// touches eight cache lines and a store meets every shared-memory bank four times.
//
// Operator side.  At plan time each canonical operator is packed as its real-form A in BF16
// hi / lo, in 16 pieces of 128 rows x 32 bytes laid out as K-major core matrices.  A warp
// bulk-copies the pieces into a small shared-memory ring and the MMA thread moves each into
// tensor memory with tcgen05.cp (no register or load/store-unit traffic), one operator ahead:
// while a chunk's MMAs run it copies whatever pieces of the next operator have landed.
//
// Epilogue.  Column entries carry the target's row offset in the tile and the reflection code,
// and every chunk is padded to a multiple of eight columns with columns that add into a spare
// row, so the drain loop has no per-column predicate; the row permutation mu is a shuffle taken
// only for the reflections that contain it (a warp-uniform branch), the sign a sign-bit flip.
//
// Roles: warps 0-3 drain the accumulators into the tile, warps 4-11 fill B (warp 4 + i: column
// blocks i and i + 8 of eight columns), warp 12 allocates tensor memory, copies the operators
// into it and issues the MMAs, warp 13 bulk-copies each chunk's column list into a ring, warp
// 14 bulk-copies the operator pieces.  Every mbarrier wait is bounded; a timeout raises the
// block's abort flag and the device error flag.
#include <cuda_bf16.h>

#include "hfmm_internal.cuh"
#include "tc_common.cuh"

namespace hfmm {

namespace {

using namespace tc;

constexpr int kSlots = 64;                       // coefficients of an order-7 expansion
constexpr int kM = 2 * kSlots;                   // rows of A / D
constexpr int kK = 2 * kSlots;                   // K
constexpr int kN = 128;                          // columns per chunk
constexpr int kKc = kK / 8;                      // core matrices along K
constexpr uint32_t kCoreBytes = 128;             // 8 rows x 16 bytes
constexpr uint32_t kSBO = kKc * kCoreBytes;      // next 8-row group
constexpr uint32_t kLBO = kCoreBytes;            // next 8-element K group
constexpr int kBElems = kN * kK;                 // BF16 elements per B part
constexpr int kStages = 2;                       // B stages / accumulators in flight
constexpr int kEpi = 128;                        // epilogue threads (warps 0-3)
constexpr int kProdWarp0 = 4;                    // producers: warps 4-11
constexpr int kMmaWarp = 12;
constexpr int kMetaWarp = 13;                    // column-list prefetch (bulk copies into a ring)
constexpr int kOpWarp = 14;                      // operator-piece prefetch
constexpr int kThreads = 15 * 32;
constexpr int kRing = 8;                         // chunks of column entries in flight
constexpr int kPieces = 16;                      // 4 KiB pieces of a packed operator
constexpr int kPieceElems = 2048;                // BF16 elements of a piece (128 rows x 16)
constexpr int kARing = 4;                        // operator pieces in flight
constexpr uint32_t kTmemCols = 512;              // 2 operator buffers (128 each) + 2 accumulators (128 each)
constexpr uint32_t kTmemAcc = 256;
constexpr uint32_t kIdesc = idesc_bf16(kM, kN);

static_assert(kM == kTsRows, "the plan encodes target rows in units of the kernel's rows");
static_assert(kN == kTsChunkCols, "the plan's chunks are the kernel's MMA width");
static_assert((int64_t)kPieces * kPieceElems == kTsOpElems, "packed operator size");

// element (r, k) of a K-major core-matrix tile with kKc core matrices per 8-row group
__device__ __forceinline__ uint32_t core_index(uint32_t r, uint32_t k) {
    return ((r >> 3) * kKc + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

// degree n and order m held by slot s
__host__ __device__ constexpr int slot_n(int s) {
    return (s & 15) < 15 - 2 * (s >> 4) ? 7 - (s >> 4) : (s >> 4);
}
__host__ __device__ constexpr int slot_m(int s) {
    return (s & 15) < 15 - 2 * (s >> 4) ? (s & 15) - (7 - (s >> 4)) : ((s & 15) - (15 - 2 * (s >> 4))) - (s >> 4);
}
// coefficient index n^2 + n + m of slot s
__host__ __device__ constexpr int slot_coef(int s) { return slot_n(s) * slot_n(s) + slot_n(s) + slot_m(s); }
// the slot of (n, -m): the reversal inside the block, same group
__host__ __device__ constexpr int slot_rev(int s) {
    return (s & 15) < 15 - 2 * (s >> 4) ? (s & ~15) | (14 - 2 * (s >> 4) - (s & 15))
                                         : (s & ~15) | (30 - 2 * (s >> 4) - (s & 15));
}
// sign of the reflection code rc (bit 0 flip x, bit 1 flip y, bit 2 flip z) on slot s: 1 = minus
__host__ __device__ constexpr int slot_neg(int s, int rc) {
    return (((rc & 1) && (slot_m(s) & 1)) ? 1 : 0) ^ (((rc & 4) && ((slot_n(s) + slot_m(s)) & 1)) ? 1 : 0);
}

struct TsShared {
    __nv_bfloat16 b[kStages][2][kBElems];  // gathered, transformed multipoles: hi, lo per stage
    alignas(128) uint16_t apiece[kARing][kPieceElems];  // operator pieces (bulk-copy targets)
    uint64_t bfull[kStages], bempty[kStages];
    uint64_t afull[kStages], aempty[kStages];
    uint64_t oempty[2];                    // the MMAs of the operator in tensor buffer b completed
    uint64_t pfull[kARing], pempty[kARing];  // operator pieces: landed / copied into tensor memory
    uint64_t mfull[kRing], mempty[kRing];  // column-entry ring: bulk copy landed / epilogue done
    uint64_t drain;
    alignas(16) int2 ring[kRing][kN];      // column entries of chunks w % kRing (bulk-copy targets)
    uint32_t tmem;
    int abort;
    // the tile's chunk records (nchunk TsChunk) and then its locals ((kTsTile + 1) x 128 floats,
    // slot order, the last row the padding columns' spare) follow
};

__host__ __device__ constexpr size_t ts_fixed_bytes() { return (sizeof(TsShared) + 127) & ~(size_t)127; }
__host__ __device__ constexpr size_t ts_chunk_bytes(int max_chunks) {
    return ((size_t)max_chunks * sizeof(TsChunk) + 127) & ~(size_t)127;
}

// Canonical operator op in the kernel's packed form: piece p (0..15) holds tensor-memory
// columns 8p .. 8p+7 of A, i.e. row r's K entries 16 (p % 8) .. +15 of part p / 8 (0 hi, 1 lo),
// as K-major core matrices (8 rows x 16 bytes; the two K halves of a row 128 bytes apart, row
// groups 256 bytes apart).  A row 2s / 2s+1 = [Re T_s, Im T_s] / [Im T_s, -Re T_s] over the
// input slots (K < 64 real part, K >= 64 imaginary part), T in slot order (plan time).
__global__ void k_ts_pack_ops(const float2* __restrict__ T, int P, int nops, uint16_t* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)nops * kTsOpElems) return;
    const int op = (int)(e / kTsOpElems), w = (int)(e % kTsOpElems);
    const int p = w / kPieceElems, q = w % kPieceElems;
    const int grp = q >> 6, ri = (q >> 3) & 7, el = q & 7;  // core matrix (row group, K half), row, element
    const int r = 8 * (grp >> 1) + ri, kc = grp & 1;
    const int K = 16 * (p & 7) + 8 * kc + el;
    const int sl = r >> 1, sl2 = K & 63;
    const int c = slot_coef(sl), c2 = slot_coef(sl2);
    const float2 t = (c < P && c2 < P) ? T[(int64_t)op * P * P + (int64_t)c * P + c2] : make_float2(0.f, 0.f);
    const float v = (r & 1) ? (K < 64 ? t.y : -t.x) : (K < 64 ? t.x : t.y);
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 x = (p < 8) ? hi : __float2bfloat16_rn(v - __bfloat162float(hi));
    out[e] = __bfloat16_as_ushort(x);
}

__device__ __forceinline__ void red_add_v2(float* p, float a, float b) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}

// out[box][v][q][o]: 16-byte row o (slots 8o .. 8o+7) of row q (0 hi Re, 1 hi -Im, 2 lo Re,
// 3 lo -Im) of the box's multipoles in slot order, v = 1 with mu applied (orders reversed)
__global__ void k_ts_split(TsSplitTable t, int64_t boxes, const float2* __restrict__ coef, uint4* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= boxes * 64) return;
    int64_t box = e >> 6;
    int l = 0;
    while (l + 1 < t.nlev && box >= t.lev[l].nbox) box -= t.lev[l++].nbox;
    const TsSplitLevel lv = t.lev[l];
    const int v = (int)(e >> 5) & 1, q = (int)(e >> 3) & 3, o = (int)e & 7;
    const float2* M = coef + lv.src + box * lv.P;
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float x[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int sl = 8 * o + 2 * j + u, ci = slot_coef(v ? slot_rev(sl) : sl);
            const float2 c = ci < lv.P ? M[ci] : make_float2(0.f, 0.f);
            x[u] = (q & 1) ? -c.y : c.x;
        }
        uint32_t hi, lo;
        split_bf16x2(x[0], x[1], hi, lo);
        w[j] = (q & 2) ? lo : hi;
    }
    out[lv.bx + box * 64 + (e & 63)] = make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ uint4 ld_nc16(const uint4* p) {
    uint4 v;
    asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// sign-bit mask of a 16-byte row of eight BF16 slots (bit e of m8: slot e negated)
__device__ __forceinline__ uint4 sign_mask(uint32_t m8) {
    uint32_t r[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) r[j] = (((m8 >> (2 * j)) & 1u) << 15) | (((m8 >> (2 * j + 1)) & 1u) << 31);
    return make_uint4(r[0], r[1], r[2], r[3]);
}

// Producer warp pw fills column blocks pw and pw + 8 (eight columns each) of every chunk's B.
// Lane (column cl = lane % 8 of the block, slot group g = lane / 8) copies the 16-byte rows of
// slots 16g .. 16g+15 in each of the four rows q, flipping the reflection's signs.
__device__ __forceinline__ void produce(TsShared& S, const TsChunk* __restrict__ ch, int nch,
                                        const uint4* __restrict__ bx, int pw, volatile int* abort, int* err) {
    const int lane = threadIdx.x & 31, cl = lane & 7, g = lane >> 3;
    uint32_t modd[2] = {0u, 0u}, nmodd[2] = {0u, 0u};  // bit e: slot 16g + 8h + e has m odd / n + m odd
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int sl = 16 * g + 8 * h + e;
            modd[h] |= (uint32_t)(slot_m(sl) & 1) << e;
            nmodd[h] |= (uint32_t)((slot_n(sl) + slot_m(sl)) & 1) << e;
        }
    for (int w = 0; w < nch; ++w) {
        const int s = w & 1;
        const uint32_t ph = (uint32_t)(w >> 1) & 1u;
        const int slot = w % kRing;
        if (!warp_wait(smem_u32(&S.mfull[slot]), (uint32_t)(w / kRing) & 1u, abort, err)) break;
        const int ncol = ch[w].ncol;
        bool ok = true;
#pragma unroll 1
        for (int i = 0; i < 2; ++i) {
            const int c = 8 * (pw + 8 * i) + cl;
            const bool on = c < ncol;
            uint4 v[8];
            int rc = 0;
            if (on) {
                const int ex = S.ring[slot][c].x;  // source box | rc << 24
                rc = (ex >> 24) & 7;
                const uint4* src = bx + (int64_t)(ex & 0xffffff) * 64 + ((rc ^ (rc >> 1)) & 1) * 32 + 2 * g;
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = ld_nc16(src + (q >> 1) * 8 + (q & 1));
            }
            // the first block's loads are in flight while the stage is awaited
            if (i == 0 && !warp_wait(smem_u32(&S.bempty[s]), ph ^ 1u, abort, err)) {
                ok = false;
                break;
            }
            if (on) {
                uint4 m[2];
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    m[h] = sign_mask(((rc & 1) ? modd[h] : 0u) ^ ((rc & 4) ? nmodd[h] : 0u));
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int row = q >> 1, h = q & 1;
                    const uint4 x = make_uint4(v[q].x ^ m[h].x, v[q].y ^ m[h].y, v[q].z ^ m[h].z, v[q].w ^ m[h].w);
                    __nv_bfloat16* base = &S.b[s][row >> 1][0];
                    *reinterpret_cast<uint4*>(base + core_index(c, 64 * (row & 1) + 16 * g + 8 * h)) = x;
                }
            }
        }
        if (!ok) break;
        fence_async_smem();  // this thread's stores -> visible to the tensor core
        mbar_arrive(smem_u32(&S.bfull[s]));
    }
}


__global__ void __launch_bounds__(kThreads, 1)
    k_m2l_ts(const TsTile* __restrict__ tiles, const TsChunk* __restrict__ chunks, const int2* __restrict__ cols,
             const uint16_t* __restrict__ canon, const uint4* __restrict__ bx, float2* __restrict__ coef,
             int* __restrict__ err, int max_chunks) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TsShared& S = *reinterpret_cast<TsShared*>(smem_raw);
    TsChunk* ch = reinterpret_cast<TsChunk*>(smem_raw + ts_fixed_bytes());  // the tile's chunk records
    float* loc = reinterpret_cast<float*>(smem_raw + ts_fixed_bytes() + ts_chunk_bytes(max_chunks));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const TsTile tile = tiles[blockIdx.x];
    const int P = tile.P;
    const int nch = tile.nchunk;
    volatile int* abort = &S.abort;

    if (warp == kMmaWarp) tmem_alloc(smem_u32(&S.tmem), kTmemCols);
    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) {
            mbar_init(smem_u32(&S.bfull[q]), (kMmaWarp - kProdWarp0) * 32);
            mbar_init(smem_u32(&S.bempty[q]), 1);
            mbar_init(smem_u32(&S.afull[q]), 1);
            mbar_init(smem_u32(&S.aempty[q]), kEpi);
        }
        for (int q = 0; q < 2; ++q) mbar_init(smem_u32(&S.oempty[q]), 1);
        for (int q = 0; q < kARing; ++q) {
            mbar_init(smem_u32(&S.pfull[q]), 1);
            mbar_init(smem_u32(&S.pempty[q]), 1);
        }
        for (int q = 0; q < kRing; ++q) {
            mbar_init(smem_u32(&S.mfull[q]), 1);
            mbar_init(smem_u32(&S.mempty[q]), kEpi);
        }
        mbar_init(smem_u32(&S.drain), 1);
        S.abort = 0;
    }
    for (int q = tid; q < nch; q += kThreads) ch[q] = chunks[tile.chunk0 + q];  // one coalesced pass
    for (int e = tid; e < tile.ntgt * kM; e += kThreads) loc[e] = 0.f;
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;

    if (warp >= kProdWarp0 && warp < kMmaWarp) {
        // ---------------------------------------------------------------- producers
        produce(S, ch, nch, bx + tile.bx, warp - kProdWarp0, abort, err);
    } else if (warp == kMmaWarp) {
        // ---------------------------------------------------------------- operator copies + MMAs
        if (lane == 0) {
            int nops = 0;
            for (int w = 0; w < nch; ++w) nops += ch[w].newop;
            int opk = -1, nc = 0;  // nc: operator pieces copied into tensor memory so far
            // piece nc (operator nc / 16, piece nc % 16) into tensor buffer (nc / 16) % 2: 1 done,
            // 0 not ready (non-blocking mode), -1 wait gave up
            auto copy_piece = [&](bool block) -> int {
                const int op = nc / kPieces, p = nc % kPieces, slot = nc % kARing;
                if (p == 0 && op >= 2) {  // the buffer's previous operator has finished its MMAs
                    const uint32_t b = smem_u32(&S.oempty[op & 1]), par = ((uint32_t)(op >> 1) & 1u) ^ 1u;
                    if (block) {
                        if (!wait_or_abort(b, par, abort, err)) return -1;
                    } else if (!mbar_test_wait(b, par)) {
                        return 0;
                    }
                }
                const uint32_t f = smem_u32(&S.pfull[slot]), fpar = (uint32_t)(nc / kARing) & 1u;
                if (block) {
                    if (!wait_or_abort(f, fpar, abort, err)) return -1;
                } else if (!mbar_test_wait(f, fpar)) {
                    return 0;
                }
                tc_fence_after();
                tc_cp_128x256(tmem + (uint32_t)((op & 1) * 128 + 8 * p),
                              umma_desc(smem_u32(&S.apiece[slot][0]), 128u, 256u));
                tc_commit(smem_u32(&S.pempty[slot]));  // the slot is free once the copy has completed
                ++nc;
                return 1;
            };
            for (int w = 0; w < nch; ++w) {
                if (ch[w].newop) {
                    ++opk;
                    int r = 1;
                    while (r > 0 && nc < kPieces * (opk + 1)) r = copy_piece(true);
                    if (r < 0) break;
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
#pragma unroll
                for (int k = 0; k < kK / 16; ++k) {
                    const uint64_t ko = (uint64_t)k * kStep;
                    const uint32_t ah = abase + (uint32_t)(8 * k), al = abase + 64u + (uint32_t)(8 * k);
                    mma_bf16_ta(d, ah, dbh + ko, kIdesc, k > 0);
                    mma_bf16_ta(d, ah, dbl + ko, kIdesc, 1);
                    mma_bf16_ta(d, al, dbh + ko, kIdesc, 1);
                }
                tc_commit(smem_u32(&S.bempty[s]));
                tc_commit(smem_u32(&S.afull[s]));
                if (w + 1 == nch || ch[w + 1].newop) tc_commit(smem_u32(&S.oempty[opk & 1]));
                // while these MMAs run: the next operator's pieces that have landed
                while (nc < kPieces * min(opk + 2, nops) && copy_piece(false) > 0) {
                }
            }
            // every tensor-core operation of this thread completes before the memory is released
            tc_commit(smem_u32(&S.drain));
            for (long long it = 0; it < kWaitLimit; ++it)
                if (mbar_try_wait(smem_u32(&S.drain), 0u)) break;
        }
        __syncwarp();
    } else if (warp == kOpWarp) {
        // ---------------------------------------------------------------- operator pieces
        if (lane == 0) {
            int n = 0;
            bool ok = true;
            for (int w = 0; w < nch && ok; ++w) {
                if (!ch[w].newop) continue;
                const uint16_t* src = canon + ch[w].op;
                for (int p = 0; p < kPieces; ++p, ++n) {
                    const int slot = n % kARing;
                    if (n >= kARing &&
                        !wait_or_abort(smem_u32(&S.pempty[slot]), ((uint32_t)(n / kARing) & 1u) ^ 1u, abort, err)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(smem_u32(&S.pfull[slot]), 2u * kPieceElems);
                    bulk_g2s(smem_u32(&S.apiece[slot][0]), src + (int64_t)p * kPieceElems, 2u * kPieceElems,
                             smem_u32(&S.pfull[slot]));
                }
            }
        }
        __syncwarp();
    } else if (warp == kMetaWarp) {
        // ---------------------------------------------------------------- column-list prefetch
        // chunk w's entries (a multiple of 8, 16-byte aligned in global memory) into ring slot w % kRing
        if (lane == 0) {
            for (int w = 0; w < nch; ++w) {
                const int slot = w % kRing;
                if (w >= kRing &&
                    !wait_or_abort(smem_u32(&S.mempty[slot]), ((uint32_t)(w / kRing) & 1u) ^ 1u, abort, err))
                    break;
                const uint32_t bytes = (uint32_t)(ch[w].ncol * sizeof(int2));
                mbar_arrive_expect_tx(smem_u32(&S.mfull[slot]), bytes);
                bulk_g2s(smem_u32(&S.ring[slot][0]), cols + ch[w].col0, bytes, smem_u32(&S.mfull[slot]));
            }
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- epilogue (warps 0..3)
        // Warp q holds rows 32q .. 32q+31, the slots of group q: thread `lane` is row
        // 2 sl + part, sl = 16q + lane / 2.  Under a reflection with mu the row's value comes
        // from the lane of the reversed slot (same warp), times this row's sign.
        const int r = tid, sl = r >> 1, part = r & 1;
        const int partner = 2 * (slot_rev(sl) & 15) + part;
        uint32_t negmask = 0;
        for (int rc = 0; rc < 8; ++rc) negmask |= (uint32_t)slot_neg(sl, rc) << rc;
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
            // the accumulator in four quarters of 32 columns, released after the last load; no
            // target repeats within an aligned group of 8 columns, so 8 are read, then written
#pragma unroll 1
            for (int hh = 0; hh < kN; hh += 32) {
                float v[32];
                tmem_ld32(acc + (uint32_t)hh, v);
                if (hh + 32 == kN) {
                    tc_fence_before();
                    mbar_arrive(smem_u32(&S.aempty[s]));
                }
                if (hh >= ncol) continue;  // warp-uniform
#pragma unroll
                for (int b8 = 0; b8 < 32; b8 += 8) {
                    if (hh + b8 < ncol) {  // warp-uniform; ncol is a multiple of 8
                        float x[8], cur[8];
                        int at[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int y = ent[hh + b8 + q].y;  // target row offset | rc << 24
                            const int rc = y >> 24;
                            float xv = v[b8 + q];
                            if ((0x66 >> rc) & 1) xv = __shfl_sync(0xffffffffu, xv, partner);  // mu: warp-uniform
                            x[q] = __int_as_float(__float_as_int(xv) ^ (int)(((negmask >> rc) & 1u) << 31));
                            at[q] = (y & 0xffffff) + r;
                            cur[q] = loc[at[q]];
                        }
#pragma unroll
                        for (int q = 0; q < 8; ++q) loc[at[q]] = cur[q] + x[q];
                    }
                }
            }
            mbar_arrive(smem_u32(&S.mempty[slot]));  // the ring slot may be refilled
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // the tile's locals into the expansion array in coefficient order (added: the locals may
    // hold other contributions)
    for (int e = tid; e < tile.ntgt * kSlots; e += kThreads) {
        const int j = e >> 6, sl = e & 63, ci = slot_coef(sl);
        if (ci < P)
            red_add_v2(reinterpret_cast<float*>(coef + tile.dst + (int64_t)j * P + ci), loc[j * kM + 2 * sl],
                       loc[j * kM + 2 * sl + 1]);
    }
    if (warp == kMmaWarp) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

size_t m2l_ts_smem(int max_chunks) {
    return ts_fixed_bytes() + ts_chunk_bytes(max_chunks) + sizeof(float) * (size_t)(kTsTile + 1) * kM;
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

void m2l_ts_pack_ops(const float2* T, int P, int nops, uint16_t* out, cudaStream_t st) {
    const int64_t n = (int64_t)nops * kTsOpElems;
    k_ts_pack_ops<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(T, P, nops, out);
    HFMM_CUDA(cudaGetLastError());
}

void m2l_ts_split(const TsSplitTable& t, int64_t boxes, const float2* coef, uint4* bx, cudaStream_t st) {
    if (boxes <= 0) return;
    k_ts_split<<<(unsigned)((boxes * 64 + 255) / 256), 256, 0, st>>>(t, boxes, coef, bx);
    HFMM_CUDA(cudaGetLastError());
}

void m2l_ts_launch(const TsTile* tiles, int64_t ntiles, int max_chunks, const TsChunk* chunks, const int2* cols,
                   const uint16_t* canon, const uint4* bx, float2* coef, int* err, cudaStream_t st) {
    if (ntiles <= 0) return;
    k_m2l_ts<<<(unsigned)ntiles, kThreads, m2l_ts_smem(max_chunks), st>>>(tiles, chunks, cols, canon, bx, coef, err,
                                                                         max_chunks);
    HFMM_CUDA(cudaGetLastError());
}

}  // namespace hfmm
