// Point sum of the Helmholtz kernel without any device allocation.
//
// For callers that cannot allocate device memory: code running where
// cudaMalloc is unavailable or forbidden (inside another library's memory
// pool, under a caller-owned arena, or in a process that must not grow its
// device footprint after start-up).  The variant stages its working set in a
// fixed file-scope __device__ array instead of plan-owned buffers; the caller
// passes only inputs and outputs.  No plan is needed.
#include <cmath>
#include <mutex>
#include <string>

#include "hfmm_internal.cuh"

namespace {

constexpr int64_t kMaxPoints = HFMM_NOALLOC_MAX_POINTS;
constexpr int kMaxDevices = 64;

// k (x - x_0) split into float32 hi + lo parts, so a difference of two nearby
// points keeps float32 relative precision however far they sit from x_0.
struct StagedSource {
    float4 hi;  // hi parts of k (x - x_0), Re (k w s / (4 pi))
    float4 lo;  // lo parts of k (x - x_0), Im (k w s / (4 pi))
};

// Shared by every call on a device and kept until the process exits
// (32 B x 262,144 = 8 MiB per device that loads the library).
static __device__ __align__(256) StagedSource g_noalloc_scratch[kMaxPoints];

std::mutex g_setup_mutex;
StagedSource* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array for the current device; looked up once
// per device with that device current (the host-side symbol is only a stand-in).
cudaError_t scratch_address(StagedSource** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<StagedSource*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// Stage positions relative to the first point (scaled by k, as hi + lo float32
// pairs) and the pre-weighted density.  Every entry [0, n) is overwritten, so
// nothing left by an earlier call is read.
__global__ void k_noalloc_stage(int64_t n, const double* __restrict__ xyz, const double* __restrict__ w,
                                const float2* __restrict__ density, double k, StagedSource* __restrict__ scratch) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double px = k * (xyz[3 * i] - xyz[0]), py = k * (xyz[3 * i + 1] - xyz[1]),
                 pz = k * (xyz[3 * i + 2] - xyz[2]);
    const float hx = (float)px, hy = (float)py, hz = (float)pz;
    float sc = (float)(k * w[i] / (4.0 * 3.14159265358979323846));
    float2 d = density[i];
    StagedSource s;
    s.hi = make_float4(hx, hy, hz, sc * d.x);
    s.lo = make_float4((float)(px - (double)hx), (float)(py - (double)hy), (float)(pz - (double)hz), sc * d.y);
    scratch[i] = s;
}

// All-pairs sum over the staged sources.  A coordinate difference is
// (hi_t - hi_s) + (lo_t - lo_s): for nearby points the first term is exact, so
// the difference carries float32 relative precision even where |k (x - x_0)|
// is large (the plain float32 difference would lose it to the offset).
__global__ void __launch_bounds__(256) k_noalloc_sum(int64_t n, const StagedSource* __restrict__ scratch,
                                                     float2* __restrict__ out) {
    __shared__ float4 shi[256];
    __shared__ float4 slo[256];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool active = i < n;
    StagedSource t = active ? scratch[i] : StagedSource{make_float4(0, 0, 0, 0), make_float4(0, 0, 0, 0)};
    float ar = 0.f, ai = 0.f;
    for (int64_t j0 = 0; j0 < n; j0 += 256) {
        int64_t j = j0 + threadIdx.x;
        if (j < n) {
            shi[threadIdx.x] = scratch[j].hi;
            slo[threadIdx.x] = scratch[j].lo;
        }
        __syncthreads();
        int cnt = (n - j0 < 256) ? (int)(n - j0) : 256;
        for (int q = 0; q < cnt; ++q) {
            if (j0 + q == i) continue;
            const float4 h = shi[q], l = slo[q];
            float dx = (t.hi.x - h.x) + (t.lo.x - l.x);
            float dy = (t.hi.y - h.y) + (t.lo.y - l.y);
            float dz = (t.hi.z - h.z) + (t.lo.z - l.z);
            float u = dx * dx + dy * dy + dz * dz;
            if (u == 0.f) continue;
            float rinv = rsqrtf(u), r = u * rinv, sn, cs;
            sincosf(r, &sn, &cs);
            float re = cs * rinv, im = sn * rinv;
            ar += h.w * re - l.w * im;
            ai += h.w * im + l.w * re;
        }
        __syncthreads();
    }
    if (active) out[i] = make_float2(ar, ai);
}

}  // namespace

extern "C" int hfmm_point_sum_noalloc(const double* xyz, const double* w, int64_t n, double k,
                                      const void* density, void* potential, void* stream) {
    if (!xyz || !w || !density || !potential) {
        hfmm_set_last_error("hfmm_point_sum_noalloc: null pointer argument");
        return HFMM_E_INVALID;
    }
    if (n <= 0) {
        hfmm_set_last_error("hfmm_point_sum_noalloc: n must be positive");
        return HFMM_E_INVALID;
    }
    if (!(k > 0.0) || !std::isfinite(k)) {
        hfmm_set_last_error("hfmm_point_sum_noalloc: k must be finite and positive");
        return HFMM_E_INVALID;
    }
    if (n > kMaxPoints) {
        hfmm_set_last_error("hfmm_point_sum_noalloc: n = " + std::to_string(n) +
                            " exceeds the scratch capacity HFMM_NOALLOC_MAX_POINTS = " + std::to_string(kMaxPoints));
        return HFMM_E_OVERFLOW;
    }
    StagedSource* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        hfmm_set_last_error(std::string("hfmm_point_sum_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return HFMM_E_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread) {
        // the scratch address is per device: the stream must belong to the current one
        int cur = 0, sdev = 0;
        e = cudaGetDevice(&cur);
        if (e == cudaSuccess) e = cudaStreamGetDevice(st, &sdev);
        if (e != cudaSuccess) {
            hfmm_set_last_error(std::string("hfmm_point_sum_noalloc: stream device: ") + cudaGetErrorString(e));
            return HFMM_E_CUDA;
        }
        if (sdev != cur) {
            hfmm_set_last_error("hfmm_point_sum_noalloc: the stream belongs to device " + std::to_string(sdev) +
                                ", not the current device " + std::to_string(cur));
            return HFMM_E_INVALID;
        }
    }
    unsigned nb = (unsigned)((n + 255) / 256);
    k_noalloc_stage<<<nb, 256, 0, st>>>(n, xyz, w, (const float2*)density, k, scratch);
    k_noalloc_sum<<<nb, 256, 0, st>>>(n, scratch, (float2*)potential);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        hfmm_set_last_error(std::string("hfmm_point_sum_noalloc: launch: ") + cudaGetErrorString(e));
        return HFMM_E_CUDA;
    }
    return HFMM_OK;
}
