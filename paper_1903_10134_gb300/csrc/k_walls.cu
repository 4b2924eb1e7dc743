// Wall construction from a voxel image (Sec. 2.3 of arXiv:1903.10134): one
// sweep marks the solid voxels within the shell thickness of the pore space,
// a second fills them with wall particles; plus the bit-packed solid mask the
// reflection test reads (Sec. 2.2).
#include "mdpd_internal.cuh"
#include "philox.cuh"

namespace mdpd {

namespace {

constexpr uint32_t WALL_TAG = 0x57414C4Cu;

__global__ void k_mask_pack(const uint8_t* __restrict__ mask, int64_t nvox,
                            uint32_t* __restrict__ bits)
{
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b = w * 32;
    if (b >= nvox) return;
    uint32_t word = 0;
    for (int k = 0; k < 32 && b + k < nvox; ++k)
        if (mask[b + k]) word |= 1u << k;
    bits[w] = word;
}

struct Dim3i {
    int v[3];
};

// count[vid] = particles of voxel vid: floor(lam + u) for shell voxels, else 0.
__global__ void k_wall_count(const uint8_t* __restrict__ mask, Dim3i dim, Dim3i per, int R,
                             int64_t R2, double lam, uint32_t key0, uint32_t key1,
                             uint32_t* __restrict__ count)
{
    const int64_t nvox = (int64_t)dim.v[0] * dim.v[1] * dim.v[2];
    const int64_t vid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (vid >= nvox) return;
    uint32_t cnt = 0;
    if (mask[vid]) {
        const int ix = (int)(vid % dim.v[0]);
        const int iy = (int)((vid / dim.v[0]) % dim.v[1]);
        const int iz = (int)(vid / ((int64_t)dim.v[0] * dim.v[1]));
        bool shell = false;
        for (int dz = -R; dz <= R && !shell; ++dz) {
            int z = iz + dz;
            if (z < 0 || z >= dim.v[2]) {
                if (!per.v[2]) continue;
                z = ((z % dim.v[2]) + dim.v[2]) % dim.v[2];
            }
            for (int dy = -R; dy <= R && !shell; ++dy) {
                int y = iy + dy;
                if (y < 0 || y >= dim.v[1]) {
                    if (!per.v[1]) continue;
                    y = ((y % dim.v[1]) + dim.v[1]) % dim.v[1];
                }
                for (int dx = -R; dx <= R; ++dx) {
                    if ((int64_t)dx * dx + (int64_t)dy * dy + (int64_t)dz * dz > R2) continue;
                    int x = ix + dx;
                    if (x < 0 || x >= dim.v[0]) {
                        if (!per.v[0]) continue;
                        x = ((x % dim.v[0]) + dim.v[0]) % dim.v[0];
                    }
                    if (!mask[x + (int64_t)dim.v[0] * (y + (int64_t)dim.v[1] * z)]) {
                        shell = true;
                        break;
                    }
                }
            }
        }
        if (shell) {
            U4 c = { (uint32_t)vid, 0u, WALL_TAG, 0u };
            const U4 w = philox4x32_10(c, key0, key1);
            const double u = __dmul_rn(__dadd_rn((double)w.x, 0.5), 2.3283064365386962890625e-10);
            cnt = (uint32_t)floor(__dadd_rn(lam, u));
        }
    }
    count[vid] = cnt;
}

__global__ void k_wall_emit(const uint32_t* __restrict__ count, const uint32_t* __restrict__ offset,
                            Dim3i dim, double voxel, double ox, double oy, double oz,
                            uint32_t key0, uint32_t key1, int64_t base, int64_t cap, Master m,
                            uint8_t wall_type)
{
    const int64_t nvox = (int64_t)dim.v[0] * dim.v[1] * dim.v[2];
    const int64_t vid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (vid >= nvox) return;
    const uint32_t cnt = count[vid];
    if (cnt == 0) return;
    const int iq[3] = { (int)(vid % dim.v[0]), (int)((vid / dim.v[0]) % dim.v[1]),
                        (int)(vid / ((int64_t)dim.v[0] * dim.v[1])) };
    const double org[3] = { ox, oy, oz };
    const uint32_t first = offset[vid];
    for (uint32_t k = 0; k < cnt; ++k) {
        U4 c = { (uint32_t)vid, k + 1u, WALL_TAG, 0u };
        const U4 w = philox4x32_10(c, key0, key1);
        const uint32_t ws[3] = { w.x, w.y, w.z };
        const int64_t i = base + first + k;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const double u = __dmul_rn(__dadd_rn((double)ws[q], 0.5), 2.3283064365386962890625e-10);
            m.x[q * cap + i] = __dadd_rn(org[q], __dmul_rn(__dadd_rn((double)iq[q], u), voxel));
            m.v[q * cap + i] = 0.0;
            m.a[q * cap + i] = 0.0;
        }
        m.id[i] = (uint32_t)i;
        m.type[i] = wall_type;
    }
}

}  // namespace

void launch_mask_pack(cudaStream_t st, const uint8_t* mask, int64_t nvox, uint32_t* bits)
{
    const int64_t words = (nvox + 31) / 32;
    if (words <= 0) return;
    k_mask_pack<<<(unsigned)((words + 255) / 256), 256, 0, st>>>(mask, nvox, bits);
}

void launch_wall_count(cudaStream_t st, const uint8_t* mask, const int dim[3], const int per[3],
                       int R, int64_t R2, double lam, uint32_t key0, uint32_t key1,
                       uint32_t* count)
{
    const int64_t nvox = (int64_t)dim[0] * dim[1] * dim[2];
    if (nvox <= 0) return;
    Dim3i d = { { dim[0], dim[1], dim[2] } }, p = { { per[0], per[1], per[2] } };
    k_wall_count<<<(unsigned)((nvox + 255) / 256), 256, 0, st>>>(mask, d, p, R, R2, lam, key0,
                                                                 key1, count);
}

void launch_wall_emit(cudaStream_t st, const uint8_t*, const int dim[3], const uint32_t* count,
                      const uint32_t* offset, double voxel, const double origin[3],
                      uint32_t key0, uint32_t key1, int64_t base, int64_t cap, const Master& m,
                      uint8_t wall_type)
{
    const int64_t nvox = (int64_t)dim[0] * dim[1] * dim[2];
    if (nvox <= 0) return;
    Dim3i d = { { dim[0], dim[1], dim[2] } };
    k_wall_emit<<<(unsigned)((nvox + 255) / 256), 256, 0, st>>>(
        count, offset, d, voxel, origin[0], origin[1], origin[2], key0, key1, base, cap, m,
        wall_type);
}

}  // namespace mdpd
