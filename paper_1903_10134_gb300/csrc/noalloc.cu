// Allocation-free density pass (mdpd_density_noalloc).
//
// Some callers cannot let a library allocate device memory: a plugin inside a
// host application that owns the whole device-memory budget and hands out only
// the input and output buffers, or a caller on a latency-critical path where
// cudaMalloc/cudaFree (which can synchronise the device) are not allowed.  For
// them this file offers one entry point that computes the local densities of a
// set of particles without allocating anything: every temporary buffer of the
// binning and density kernels lives in one file-scope __device__ array of fixed
// size (below), which each GPU that loads the library keeps until the process
// exits.
//
// Host code may not use the array's name as a device address (in host code it
// names a host-side stand-in).  The device address is looked up with
// cudaGetSymbolAddress, with the device current, on every call made outside
// stream capture (so a cudaDeviceReset between calls leaves no stale address);
// a call made while its stream is being captured reuses the address of the
// last uncaptured call on that device, so the first call on a device should
// happen before any stream capture.  All calls share the array and it keeps the previous call's contents,
// so the counters that must start at zero are cleared on every call, and calls
// whose work overlaps on the GPU (on different streams, or from several host
// threads without ordering) race on the array and give wrong results.
#include <math_constants.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "f64bits.cuh"
#include "mdpd_internal.cuh"
#include "vec.cuh"

namespace mdpd {

void set_global_error(const std::string& msg);

namespace {

constexpr int64_t NA_MAX_PARTICLES = 65536;
constexpr int64_t NA_MAX_CELLS = 32768;
constexpr size_t NA_ALIGN = 256;

constexpr size_t na_round(size_t b) { return (b + NA_ALIGN - 1) / NA_ALIGN * NA_ALIGN; }

// Byte offsets of the parts of the scratch array.
constexpr size_t OFF_COUNT = 0;
constexpr size_t OFF_START = OFF_COUNT + na_round(NA_MAX_CELLS * 4);
constexpr size_t OFF_SCAN = OFF_START + na_round((NA_MAX_CELLS + 1) * 4);
constexpr size_t OFF_CELLOF = OFF_SCAN + na_round(64 * 4);
constexpr size_t OFF_SLOT = OFF_CELLOF + na_round(NA_MAX_PARTICLES * 4);
constexpr size_t OFF_KEY = OFF_SLOT + na_round(NA_MAX_PARTICLES * 4);
constexpr size_t OFF_SRC = OFF_KEY + na_round(NA_MAX_PARTICLES * 4);
constexpr size_t OFF_CELLS = OFF_SRC + na_round(NA_MAX_PARTICLES * 4);
constexpr size_t OFF_POS4 = OFF_CELLS + na_round(NA_MAX_PARTICLES * 4);
constexpr size_t OFF_RHO = OFF_POS4 + na_round(NA_MAX_PARTICLES * sizeof(D4));
constexpr size_t NA_BYTES = OFF_RHO + na_round(NA_MAX_PARTICLES * sizeof(double));

// The scratch memory (about 4.3 MB).
static __device__ __align__(256) unsigned char g_na_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
void* g_na_ptr[NA_MAX_DEVICES] = {};

// Device address of the scratch array on the current device.  Outside stream
// capture it is looked up on every call (a lookup allocates nothing), so a
// cudaDeviceReset or a new primary context between calls cannot leave a
// stale address behind; while the stream is being captured the address
// recorded by the last uncaptured call on this device is used, and a call
// that has none is refused.
int scratch_address(cudaStream_t st, void** out, std::string& why)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        why = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return MDPD_ERR_CUDA;
    }
    if (dev < 0 || dev >= NA_MAX_DEVICES) {
        why = "device index out of range for the scratch table";
        return MDPD_ERR_INVALID_ARG;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) {
        why = std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e);
        return MDPD_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess || !p) {
            why = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return MDPD_ERR_CUDA;
        }
        g_na_ptr[dev] = p;
    } else if (!g_na_ptr[dev]) {
        why = "the first call on a device must come before any stream capture";
        return MDPD_ERR_INVALID_ARG;
    }
    *out = g_na_ptr[dev];
    return MDPD_OK;
}

// Whether position x lies outside the box on a non-periodic axis (the closed
// upper face is accepted: a particle on it is binned into the last cell, where
// the search of the neighbouring cells stays complete), or is not finite.
__device__ __forceinline__ bool na_outside(const double* __restrict__ x, const Geo& geo)
{
    bool out = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (!isfinite(x[k])) out = true;
        else if (!geo.periodic[k] && (x[k] < geo.lo[k] || x[k] > geo.hi[k])) out = true;
    }
    return out;
}

__global__ void k_na_count(int n, const double* __restrict__ pos, Geo geo,
                           uint32_t* __restrict__ cellof, uint32_t* __restrict__ slot,
                           uint32_t* __restrict__ count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double x = pos[3 * (int64_t)i + k];
        if (geo.periodic[k]) x -= geo.L[k] * floor((x - geo.lo[k]) / geo.L[k]);
        int c = (int)floor((x - geo.lo[k]) * geo.inv_h[k]);
        q[k] = c < 0 ? 0 : (c >= geo.nc[k] ? geo.nc[k] - 1 : c);
    }
    const uint32_t c = (uint32_t)(q[0] + geo.nc[0] * (q[1] + geo.nc[1] * q[2]));
    cellof[i] = c;
    slot[i] = atomicAdd(&count[c], 1u);
}

__global__ void k_na_scatter(int n, const uint32_t* __restrict__ cellof,
                             const uint32_t* __restrict__ slot, const uint32_t* __restrict__ start,
                             uint32_t* __restrict__ key, uint32_t* __restrict__ src)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t d = start[cellof[i]] + slot[i];
    key[d] = (uint32_t)i;
    src[d] = (uint32_t)i;
}

template <typename T>
__global__ void k_na_gather(int n, const double* __restrict__ pos, const uint32_t* __restrict__ src,
                            const uint32_t* __restrict__ cellof, Geo geo,
                            typename Vec4<T>::type* __restrict__ pos4, uint32_t* __restrict__ cell_s)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t i = src[s];
    const uint32_t c = cellof[i];
    const int q[3] = { (int)(c % (uint32_t)geo.nc[0]),
                       (int)((c / (uint32_t)geo.nc[0]) % (uint32_t)geo.nc[1]),
                       (int)(c / ((uint32_t)geo.nc[0] * (uint32_t)geo.nc[1])) };
    T off[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double x = pos[3 * (int64_t)i + k];
        if (geo.periodic[k]) x -= geo.L[k] * floor((x - geo.lo[k]) / geo.L[k]);
        off[k] = (T)(x - geo.lo[k] - ((double)q[k] + 0.5) * geo.h[k]);
    }
    pos4[s] = make4(off[0], off[1], off[2], pack_u32(T(0), 0u));
    cell_s[s] = c;
}

// Densities back to input order; a particle outside the box on a
// non-periodic axis (or with a non-finite coordinate) gets NaN, so a bad
// input shows in the output instead of as a silently clamped cell.
template <typename T>
__global__ void k_na_unsort(int n, const double* __restrict__ pos, Geo geo,
                            const uint32_t* __restrict__ src, const T* __restrict__ r,
                            double* __restrict__ out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t i = src[s];
    out[i] = na_outside(pos + 3 * (int64_t)i, geo) ? CUDART_NAN : (double)r[s];
}

}  // namespace

}  // namespace mdpd

using namespace mdpd;

extern "C" int mdpd_density_noalloc(const mdpd_params* p, int64_t n, const double* pos,
                                    double* rho, void* cuda_stream)
{
    std::string why;
    auto bad = [&](int code, const std::string& msg) -> int {
        set_global_error("mdpd_density_noalloc: " + msg);
        return code;
    };
    if (!p) return bad(MDPD_ERR_INVALID_ARG, "params is NULL");
    if (n < 0 || n > NA_MAX_PARTICLES)
        return bad(MDPD_ERR_INVALID_ARG, "n must be in 0.." + std::to_string(NA_MAX_PARTICLES));
    if (n > 0 && (!pos || !rho)) return bad(MDPD_ERR_INVALID_ARG, "pos and rho are required");
    if (!(p->rc > 0) || !(p->rd > 0) || !(p->rd <= p->rc) || !std::isfinite(p->rc))
        return bad(MDPD_ERR_INVALID_ARG, "need 0 < rd <= rc");
    if (p->precision != 0 && p->precision != 1)
        return bad(MDPD_ERR_INVALID_ARG, "precision must be 0 or 1");
    Geo geo{};
    geo.ncell = 1;
    for (int k = 0; k < 3; ++k) {
        if (!(p->box[k] > 0) || !std::isfinite(p->box[k]) || !std::isfinite(p->box_lo[k]))
            return bad(MDPD_ERR_INVALID_ARG, "box lengths must be finite and > 0");
        if (p->periodic[k] && p->box[k] < 3.0 * p->rc)
            return bad(MDPD_ERR_INVALID_ARG, "a periodic axis must be at least 3 rc long");
        int m = (int)std::floor(p->box[k] / p->rc);
        if (m < 1) m = 1;
        geo.nc[k] = m;
        geo.periodic[k] = p->periodic[k] ? 1 : 0;
        geo.lo[k] = p->box_lo[k];
        geo.L[k] = p->box[k];
        geo.hi[k] = p->box_lo[k] + p->box[k];
        geo.key_lo[k] = f64_key(geo.lo[k]);
        geo.key_hi[k] = f64_key(geo.hi[k]);
        geo.h[k] = p->box[k] / m;
        geo.inv_h[k] = 1.0 / geo.h[k];
        geo.ncell *= m;
        if (geo.ncell > NA_MAX_CELLS)
            return bad(MDPD_ERR_INVALID_ARG,
                       "box has more than " + std::to_string(NA_MAX_CELLS) + " cells of edge rc");
    }
    Phys ph{};
    ph.rc = p->rc;
    ph.rd = p->rd;
    ph.rho_self = p->rho_self ? 1 : 0;
    fill_derived(ph, geo);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // an error left by earlier, unrelated work is not this call's: report it
    // without clearing it
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess)
        return bad(MDPD_ERR_CUDA, std::string("a CUDA error was pending before the call: ") +
                                      cudaGetErrorString(e));
    void* base = nullptr;
    int rc = scratch_address(st, &base, why);
    if (rc) return bad(rc, why);
    if (n == 0) return MDPD_OK;

    unsigned char* b = (unsigned char*)base;
    uint32_t* count = (uint32_t*)(b + OFF_COUNT);
    uint32_t* start = (uint32_t*)(b + OFF_START);
    uint32_t* scan = (uint32_t*)(b + OFF_SCAN);
    uint32_t* cellof = (uint32_t*)(b + OFF_CELLOF);
    uint32_t* slot = (uint32_t*)(b + OFF_SLOT);
    uint32_t* key = (uint32_t*)(b + OFF_KEY);
    uint32_t* src = (uint32_t*)(b + OFF_SRC);
    uint32_t* cells = (uint32_t*)(b + OFF_CELLS);
    void* pos4 = b + OFF_POS4;
    void* rs = b + OFF_RHO;
    const int nn = (int)n;
    const unsigned nb = (unsigned)((n + 255) / 256);
    // the first failing step names itself (launch errors are this call's own,
    // so they are cleared after being read)
    auto check = [&](const char* what) -> int {
        const cudaError_t le = cudaPeekAtLastError();
        if (le == cudaSuccess) return MDPD_OK;
        cudaGetLastError();
        return bad(MDPD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(le));
    };
    e = cudaMemsetAsync(count, 0, (size_t)geo.ncell * sizeof(uint32_t), st);
    if (e != cudaSuccess) return bad(MDPD_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    k_na_count<<<nb, 256, 0, st>>>(nn, pos, geo, cellof, slot, count);
    if ((rc = check("k_na_count"))) return rc;
    launch_exclusive_scan(st, count, geo.ncell, start, scan);
    if ((rc = check("cell-count scan"))) return rc;
    k_na_scatter<<<nb, 256, 0, st>>>(nn, cellof, slot, start, key, src);
    if ((rc = check("k_na_scatter"))) return rc;
    launch_cell_sort(st, geo.ncell, start, key, src, count);
    if ((rc = check("cell sort"))) return rc;
    if (p->precision == 0)
        k_na_gather<double><<<nb, 256, 0, st>>>(nn, pos, src, cellof, geo, (D4*)pos4, cells);
    else
        k_na_gather<float><<<nb, 256, 0, st>>>(nn, pos, src, cellof, geo, (float4*)pos4, cells);
    if ((rc = check("k_na_gather"))) return rc;
    launch_density(st, p->precision, nn, geo, ph, pos4, cells, start, rs);
    if ((rc = check("density pass"))) return rc;
    if (p->precision == 0)
        k_na_unsort<double><<<nb, 256, 0, st>>>(nn, pos, geo, src, (const double*)rs, rho);
    else
        k_na_unsort<float><<<nb, 256, 0, st>>>(nn, pos, geo, src, (const float*)rs, rho);
    return check("k_na_unsort");
}
