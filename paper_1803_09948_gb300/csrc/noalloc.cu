// Point sum of the Helmholtz kernel without any device allocation.
//
// For callers that cannot allocate device memory: code running where
// cudaMalloc is unavailable or forbidden (inside another library's memory
// pool, under a caller-owned arena, or in a process that must not grow its
// device footprint after start-up).  The variant stages its working set in a
// fixed file-scope __device__ array instead of plan-owned buffers; the caller
// passes only inputs and outputs.  No plan is needed.
#include <mutex>
#include <string>

#include "hfmm_internal.cuh"

namespace {

constexpr int64_t kMaxPoints = HFMM_NOALLOC_MAX_POINTS;
constexpr int kMaxDevices = 64;

struct StagedSource {
    float4 pos;  // k * (x - x_0), float32
    float2 sig;  // k w s / (4 pi)
    float2 pad;
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

// Stage positions relative to the first point (scaled by k) and the
// pre-weighted density.  Every entry [0, n) is overwritten, so nothing left by
// an earlier call is read.
__global__ void k_noalloc_stage(int64_t n, const double* __restrict__ xyz, const double* __restrict__ w,
                                const float2* __restrict__ density, double k, StagedSource* __restrict__ scratch) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double c0 = xyz[0], c1 = xyz[1], c2 = xyz[2];
    StagedSource s;
    s.pos = make_float4((float)(k * (xyz[3 * i] - c0)), (float)(k * (xyz[3 * i + 1] - c1)),
                        (float)(k * (xyz[3 * i + 2] - c2)), 0.f);
    float sc = (float)(k * w[i] / (4.0 * 3.14159265358979323846));
    float2 d = density[i];
    s.sig = make_float2(sc * d.x, sc * d.y);
    s.pad = make_float2(0.f, 0.f);
    scratch[i] = s;
}

// All-pairs sum over the staged sources (same arithmetic as the library's
// direct-summation kernel, without its leaf-local coordinates).
__global__ void __launch_bounds__(256) k_noalloc_sum(int64_t n, const StagedSource* __restrict__ scratch,
                                                     float2* __restrict__ out) {
    __shared__ float4 sp[256];
    __shared__ float2 sg[256];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool active = i < n;
    float4 t = active ? scratch[i].pos : make_float4(0, 0, 0, 0);
    float ar = 0.f, ai = 0.f;
    for (int64_t j0 = 0; j0 < n; j0 += 256) {
        int64_t j = j0 + threadIdx.x;
        if (j < n) {
            sp[threadIdx.x] = scratch[j].pos;
            sg[threadIdx.x] = scratch[j].sig;
        }
        __syncthreads();
        int cnt = (n - j0 < 256) ? (int)(n - j0) : 256;
        for (int q = 0; q < cnt; ++q) {
            if (j0 + q == i) continue;
            float4 s = sp[q];
            float dx = t.x - s.x, dy = t.y - s.y, dz = t.z - s.z;
            float u = dx * dx + dy * dy + dz * dz;
            if (u == 0.f) continue;
            float rinv = rsqrtf(u), r = u * rinv, sn, cs;
            sincosf(r, &sn, &cs);
            float re = cs * rinv, im = sn * rinv;
            float2 g = sg[q];
            ar += g.x * re - g.y * im;
            ai += g.x * im + g.y * re;
        }
        __syncthreads();
    }
    if (active) out[i] = make_float2(ar, ai);
}

}  // namespace

extern "C" int hfmm_point_sum_noalloc(const double* xyz, const double* w, int64_t n, double k,
                                      const void* density, void* potential, void* stream) {
    if (!xyz || !w || !density || !potential || n <= 0 || !(k > 0.0)) return HFMM_E_INVALID;
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
