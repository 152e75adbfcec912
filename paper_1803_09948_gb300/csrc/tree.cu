// Octree construction on the device (Sec. 2.3 octree; Sec. 3.1-3.2 Morton order, a
// cell = first index + count): Morton keys of the points and their stable sort,
// per-point leaf data (positions relative to the leaf centre, pre-scaled weights,
// integer coordinates), the 27-box neighbour lists of the leaves of a uniform tree, and
// the M2L interaction lists of one level bucketed by translation offset.
//
// Keys interleave 20 bits per axis (x in the highest bit of each triple).  Every
// list comes out in the order a sequential loop would produce it (neighbours by
// (dx, dy, dz) lexicographic, interaction pairs by offset slot and then by target
// box), so the work items built from them do not depend on thread scheduling.
#include <cub/device/device_radix_sort.cuh>

#include <vector>

#include "hfmm_internal.cuh"

namespace hfmm {

namespace {

constexpr int kLmax = 20;
constexpr int kChunk = 256;   // targets per block in the interaction-list kernels
constexpr int kSlots = 316;   // offsets in [-3,3]^3 that are not neighbours

__device__ __forceinline__ uint64_t t_spread3(uint64_t v) {
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffull;
    v = (v | v << 16) & 0x1f0000ff0000ffull;
    v = (v | v << 8) & 0x100f00f00f00f00full;
    v = (v | v << 4) & 0x10c30c30c30c30c3ull;
    v = (v | v << 2) & 0x1249249249249249ull;
    return v;
}
__device__ __forceinline__ uint64_t t_compact3(uint64_t v) {
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffff;
    return v;
}
__device__ __forceinline__ uint64_t t_morton(int64_t x, int64_t y, int64_t z) {
    return (t_spread3((uint64_t)x) << 2) | (t_spread3((uint64_t)y) << 1) | t_spread3((uint64_t)z);
}
__device__ __forceinline__ int4 t_demorton(uint64_t k) {
    return make_int4((int)t_compact3(k >> 2), (int)t_compact3(k >> 1), (int)t_compact3(k), 0);
}
// index of key in keys[0, n), or -1
__device__ __forceinline__ int64_t t_find(const uint64_t* __restrict__ keys, int64_t n, uint64_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < n && keys[lo] == key) ? lo : -1;
}

__global__ void k_morton_keys(const double* __restrict__ x, int64_t N, double lo0, double lo1, double lo2,
                              double scale, uint64_t* __restrict__ keys, int32_t* __restrict__ idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double lo[3] = {lo0, lo1, lo2};
    int64_t c[3];
    for (int d = 0; d < 3; ++d) {
        int64_t q = (int64_t)floor((x[3 * i + d] - lo[d]) * scale);
        c[d] = max((int64_t)0, min(q, ((int64_t)1 << kLmax) - 1));
    }
    keys[i] = t_morton(c[0], c[1], c[2]);
    idx[i] = (int32_t)i;
}

// one thread per sorted point: its leaf's data and the sorted copies of its inputs
__global__ void k_leaf_data(const double* __restrict__ x, const double* __restrict__ w, const int32_t* __restrict__ tri,
                            const int32_t* __restrict__ perm, const uint64_t* __restrict__ keys, int L,
                            const int4* __restrict__ leaf_c2, const int32_t* __restrict__ leaf_start, int64_t nleaf,
                            int64_t N, double lo0, double lo1, double lo2, double half_side, double k, LeafData o) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    // leaf of point i: the last b with leaf_start[b] <= i
    int64_t lo = 0, hi = nleaf - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (leaf_start[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    const int64_t b = lo;
    const int4 c = leaf_c2[b];
    const double ctr[3] = {lo0 + (double)c.x * half_side, lo1 + (double)c.y * half_side, lo2 + (double)c.z * half_side};
    const int32_t u = perm[i];
    const double xu[3] = {x[3 * (int64_t)u], x[3 * (int64_t)u + 1], x[3 * (int64_t)u + 2]};
    o.pts[i] = make_float4((float)(k * (xu[0] - ctr[0])), (float)(k * (xu[1] - ctr[1])), (float)(k * (xu[2] - ctr[2])),
                           0.f);
    o.wscale[i] = (float)(k * w[u] / (4.0 * 3.14159265358979323846));
    o.pt_leaf[i] = (int32_t)b;
    o.pt_ijk[i] = t_demorton(keys[i] >> (3 * (kLmax - L)));
    for (int d = 0; d < 3; ++d) o.x64s[3 * i + d] = xu[d];
    o.w64s[i] = w[u];
    o.tri_s[i] = tri[u];
    o.iperm[u] = (int32_t)i;
}

// neighbour lists: pass 0 counts, pass 1 writes (order dx, dy, dz) and each leaf's
// neighbourhood point count
__global__ void k_leaf_nbr(const uint64_t* __restrict__ leaf_key, const int32_t* __restrict__ leaf_start, int64_t nleaf,
                           int L, const int32_t* __restrict__ ptr, int32_t* __restrict__ cnt_or_nbr,
                           int64_t* __restrict__ hood) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    const int4 c = t_demorton(leaf_key[b]);
    const int64_t nl = (int64_t)1 << L;
    int n = 0;
    int64_t tot = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                const int64_t x = c.x + dx, y = c.y + dy, z = c.z + dz;
                if (x < 0 || y < 0 || z < 0 || x >= nl || y >= nl || z >= nl) continue;
                const int64_t s = t_find(leaf_key, nleaf, t_morton(x, y, z));
                if (s < 0) continue;
                if (ptr) {
                    cnt_or_nbr[ptr[b] + n] = (int32_t)s;
                    tot += leaf_start[s + 1] - leaf_start[s];
                }
                ++n;
            }
    if (!ptr) cnt_or_nbr[b] = n;
    else hood[b] = tot;
}

// Interaction list of target box t at one level: the children of its parent's
// neighbours that are not its own neighbours.  f(slot, source) is called for each,
// in the order (parent neighbour ex, ey, ez; child octant).
template <typename F>
__device__ __forceinline__ void for_each_vlist(const uint64_t* __restrict__ key, int64_t nbox, int l, int64_t t,
                                               const int16_t* __restrict__ slot, F&& f) {
    const int4 c = t_demorton(key[t]);
    const int64_t nlv = (int64_t)1 << l;
    const int64_t px = c.x >> 1, py = c.y >> 1, pz = c.z >> 1;
    for (int ex = -1; ex <= 1; ++ex)
        for (int ey = -1; ey <= 1; ++ey)
            for (int ez = -1; ez <= 1; ++ez) {
                const int64_t qx = px + ex, qy = py + ey, qz = pz + ez;
                if (qx < 0 || qy < 0 || qz < 0 || 2 * qx >= nlv || 2 * qy >= nlv || 2 * qz >= nlv) continue;
                // the children of parent box q are consecutive in the sorted keys
                const uint64_t qk = t_morton(qx, qy, qz) << 3;
                int64_t lo = 0, hi = nbox;
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (key[mid] < qk) lo = mid + 1;
                    else hi = mid;
                }
                for (int64_t s = lo; s < nbox && (key[s] >> 3) == (qk >> 3); ++s) {
                    const int o = (int)(key[s] & 7);
                    const int64_t dx = 2 * qx + ((o >> 2) & 1) - c.x, dy = 2 * qy + ((o >> 1) & 1) - c.y,
                                  dz = 2 * qz + (o & 1) - c.z;
                    if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1) continue;
                    f((int)slot[(dx + 3) * 49 + (dy + 3) * 7 + (dz + 3)], s);
                }
            }
}

// Marks which targets of this block's chunk have a source at each slot (one bit per
// target); every target has at most one source per slot.
__device__ __forceinline__ void vlist_flags(const uint64_t* __restrict__ key, int64_t nbox, int l,
                                            const int16_t* __restrict__ slot, uint32_t (*flags)[kChunk / 32]) {
    for (int q = threadIdx.x; q < kSlots * (kChunk / 32); q += blockDim.x) flags[q / (kChunk / 32)][q % (kChunk / 32)] = 0;
    __syncthreads();
    const int64_t t = (int64_t)blockIdx.x * kChunk + threadIdx.x;
    const int tl = threadIdx.x;
    if (t < nbox)
        for_each_vlist(key, nbox, l, t, slot,
                       [&](int g, int64_t) { atomicOr(&flags[g][tl >> 5], 1u << (tl & 31)); });
    __syncthreads();
}

__global__ void __launch_bounds__(kChunk) k_vlist_count(const uint64_t* __restrict__ key, int64_t nbox, int l,
                                                        const int16_t* __restrict__ slot, int32_t* __restrict__ cnt) {
    __shared__ uint32_t flags[kSlots][kChunk / 32];
    vlist_flags(key, nbox, l, slot, flags);
    for (int g = threadIdx.x; g < kSlots; g += blockDim.x) {
        int n = 0;
        for (int wd = 0; wd < kChunk / 32; ++wd) n += __popc(flags[g][wd]);
        cnt[(int64_t)blockIdx.x * kSlots + g] = n;
    }
}

// pair (source, target) to off[chunk][slot] + (targets of the chunk before t with that slot)
__global__ void __launch_bounds__(kChunk) k_vlist_fill(const uint64_t* __restrict__ key, int64_t nbox, int l,
                                                       const int16_t* __restrict__ slot,
                                                       const int64_t* __restrict__ off, int2* __restrict__ pairs) {
    __shared__ uint32_t flags[kSlots][kChunk / 32];
    vlist_flags(key, nbox, l, slot, flags);
    const int64_t t = (int64_t)blockIdx.x * kChunk + threadIdx.x;
    const int tl = threadIdx.x;
    if (t >= nbox) return;
    const int64_t* o = off + (int64_t)blockIdx.x * kSlots;
    for_each_vlist(key, nbox, l, t, slot, [&](int g, int64_t s) {
        int rank = __popc(flags[g][tl >> 5] & ((1u << (tl & 31)) - 1u));
        for (int wd = 0; wd < (tl >> 5); ++wd) rank += __popc(flags[g][wd]);
        pairs[o[g] + rank] = make_int2((int)s, (int)t);
    });
}

}  // namespace

void tree_sort_points(const double* x, int64_t N, const double lo[3], double scale, uint64_t* keys_sorted,
                      int32_t* perm, cudaStream_t st) {
    if (N <= 0) return;
    DBuf<uint64_t> keys;
    DBuf<int32_t> idx;
    keys.alloc(N, nullptr);
    idx.alloc(N, nullptr);
    k_morton_keys<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(x, N, lo[0], lo[1], lo[2], scale, keys.p, idx.p);
    HFMM_CUDA(cudaGetLastError());
    // LSD radix sort: stable, so equal keys keep ascending point index
    size_t tb = 0;
    HFMM_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, keys.p, keys_sorted, idx.p, perm, (int)N, 0, 3 * kLmax, st));
    DBuf<unsigned char> tmp;
    tmp.alloc(tb, nullptr);
    HFMM_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, tb, keys.p, keys_sorted, idx.p, perm, (int)N, 0, 3 * kLmax, st));
    HFMM_CUDA(cudaStreamSynchronize(st));  // the scratch buffers are freed on return
}

void tree_leaf_data(const double* x, const double* w, const int32_t* tri, const int32_t* perm, const uint64_t* keys,
                    int L, const int4* leaf_c2, const int32_t* leaf_start, int64_t nleaf, int64_t N,
                    const double lo[3], double half_side, double k, const LeafData& o, cudaStream_t st) {
    if (N <= 0) return;
    k_leaf_data<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(x, w, tri, perm, keys, L, leaf_c2, leaf_start, nleaf, N,
                                                             lo[0], lo[1], lo[2], half_side, k, o);
    HFMM_CUDA(cudaGetLastError());
}

void tree_leaf_neighbours(const uint64_t* leaf_key, const int32_t* leaf_start, int64_t nleaf, int L,
                          DBuf<int32_t>& nbr_ptr, DBuf<int32_t>& nbr, std::vector<int32_t>& h_ptr,
                          std::vector<int64_t>& h_hood, size_t* bytes, cudaStream_t st) {
    const unsigned nb = (unsigned)((nleaf + 127) / 128);
    DBuf<int32_t> cnt;
    cnt.alloc(nleaf, nullptr);
    k_leaf_nbr<<<nb, 128, 0, st>>>(leaf_key, leaf_start, nleaf, L, nullptr, cnt.p, nullptr);
    HFMM_CUDA(cudaGetLastError());
    std::vector<int32_t> c(nleaf);
    HFMM_CUDA(cudaMemcpyAsync(c.data(), cnt.p, sizeof(int32_t) * nleaf, cudaMemcpyDeviceToHost, st));
    HFMM_CUDA(cudaStreamSynchronize(st));
    h_ptr.assign(nleaf + 1, 0);
    for (int64_t b = 0; b < nleaf; ++b) h_ptr[b + 1] = h_ptr[b] + c[b];
    nbr_ptr.upload(h_ptr, bytes, st);
    nbr.alloc((size_t)std::max<int32_t>(h_ptr[nleaf], 1), bytes);
    DBuf<int64_t> hood;
    hood.alloc(nleaf, nullptr);
    k_leaf_nbr<<<nb, 128, 0, st>>>(leaf_key, leaf_start, nleaf, L, nbr_ptr.p, nbr.p, hood.p);
    HFMM_CUDA(cudaGetLastError());
    h_hood.resize(nleaf);
    HFMM_CUDA(cudaMemcpyAsync(h_hood.data(), hood.p, sizeof(int64_t) * nleaf, cudaMemcpyDeviceToHost, st));
    HFMM_CUDA(cudaStreamSynchronize(st));
}

int64_t tree_m2l_lists(const uint64_t* key, int64_t nbox, int l, const int16_t* slot, std::vector<int2>& pairs,
                       std::vector<int64_t>& bstart, cudaStream_t st) {
    bstart.assign(kSlots + 1, 0);
    pairs.clear();
    if (nbox <= 0) return 0;
    const int64_t nch = (nbox + kChunk - 1) / kChunk;
    DBuf<int32_t> cnt;
    cnt.alloc(nch * kSlots, nullptr);
    k_vlist_count<<<(unsigned)nch, kChunk, 0, st>>>(key, nbox, l, slot, cnt.p);
    HFMM_CUDA(cudaGetLastError());
    std::vector<int32_t> c(nch * kSlots);
    HFMM_CUDA(cudaMemcpyAsync(c.data(), cnt.p, sizeof(int32_t) * c.size(), cudaMemcpyDeviceToHost, st));
    HFMM_CUDA(cudaStreamSynchronize(st));
    // bucket g holds its pairs chunk by chunk: off[chunk][g] = start of g + pairs of g in earlier chunks
    std::vector<int64_t> off(nch * kSlots);
    for (int g = 0; g < kSlots; ++g) {
        int64_t run = bstart[g];
        for (int64_t ch = 0; ch < nch; ++ch) {
            off[ch * kSlots + g] = run;
            run += c[ch * kSlots + g];
        }
        bstart[g + 1] = run;
    }
    const int64_t n = bstart[kSlots];
    if (n == 0) return 0;
    DBuf<int64_t> d_off;
    d_off.upload(off, nullptr, st);
    DBuf<int2> d_pairs;
    d_pairs.alloc(n, nullptr);
    k_vlist_fill<<<(unsigned)nch, kChunk, 0, st>>>(key, nbox, l, slot, d_off.p, d_pairs.p);
    HFMM_CUDA(cudaGetLastError());
    pairs.resize(n);
    HFMM_CUDA(cudaMemcpyAsync(pairs.data(), d_pairs.p, sizeof(int2) * n, cudaMemcpyDeviceToHost, st));
    HFMM_CUDA(cudaStreamSynchronize(st));
    return n;
}

}  // namespace hfmm
