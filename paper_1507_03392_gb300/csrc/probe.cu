// Moment probes and screens: on-demand diagnostics over a run's particles as
// they are (Sec. III.A).  One pass reads each particle's fixed-point position,
// velocity and state word and
//  - adds its count and its velocity sums (v and v^2 by component, FP64) to
//    the (cell, Q) slot when its nearest-grid-point cell is probed;
//  - counts a hit on the pixel under it, by Q, for every screen whose slab
//    z_lo <= z < z_hi contains it.
// The slab test and the pixel are taken on the fixed-point coordinates: with
// U = X + 2^31 the pixel is the top log2(pixels) bits of U, so pixel edges
// fall exactly at -R0 + 2 R0 k / pixels; the cell is the same NGP cell the
// deposit uses.  Frozen particles and padding slots are skipped.
#include "ecris_internal.cuh"

namespace ecris {

namespace {

__global__ void __launch_bounds__(256) k_probe(const __grid_constant__ RunDev R, const __grid_constant__ ProbeDev P,
                                               uint32_t n4)
{
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n4; g += gridDim.x * blockDim.x) {
        const uint4 m4 = reinterpret_cast<const uint4*>(R.meta)[g];
        const uint32_t mm[4] = {m4.x, m4.y, m4.z, m4.w};
        const int4 x4 = reinterpret_cast<const int4*>(R.x)[g];
        const int4 y4 = reinterpret_cast<const int4*>(R.y)[g];
        const int4 z4 = reinterpret_cast<const int4*>(R.z)[g];
        const int32_t xs[4] = {x4.x, x4.y, x4.z, x4.w};
        const int32_t ys[4] = {y4.x, y4.y, y4.z, y4.w};
        const int32_t zs[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t meta = mm[j];
            if (meta & (kStFrozen | kStPad)) continue;
            const uint32_t Q = meta & kQMask;
            if (P.slot) {
                const int32_t s = P.slot[ngp_cell(R, xs[j], ys[j], zs[j])];
                if (s >= 0) {
                    const uint32_t i = 4 * g + j;
                    const double vx = R.vx[i], vy = R.vy[i], vz = R.vz[i];
                    double* a = P.mom + ((size_t)s * P.qs + Q) * 7;
                    atomicAdd(a + 0, 1.0);
                    atomicAdd(a + 1, vx);
                    atomicAdd(a + 2, vy);
                    atomicAdd(a + 3, vz);
                    atomicAdd(a + 4, vx * vx);
                    atomicAdd(a + 5, vy * vy);
                    atomicAdd(a + 6, vz * vz);
                }
            }
            const uint32_t u = (uint32_t)zs[j] ^ 0x80000000u;
            for (int k = 0; k < P.nscreens; ++k) {
                if (u < P.ulo[k] || u > P.uhi[k]) continue;
                const uint32_t px = ((uint32_t)xs[j] ^ 0x80000000u) >> (32 - P.pix_log2);
                const uint32_t py = ((uint32_t)ys[j] ^ 0x80000000u) >> (32 - P.pix_log2);
                const size_t plane = (size_t)(k * P.qs + (int)Q) << (2 * P.pix_log2);
                atomicAdd(P.screen + plane + ((size_t)py << P.pix_log2) + px, 1ull);
            }
        }
    }
}

}  // namespace

cudaError_t launch_probe(const RunDev& R, const ProbeDev& P, uint32_t n4, int sm_count, cudaStream_t s)
{
    if (n4 == 0) return cudaSuccess;
    const uint32_t need = (n4 + 255) / 256;
    const uint32_t blocks = need < (uint32_t)(4 * sm_count) ? need : (uint32_t)(4 * sm_count);
    k_probe<<<blocks, 256, 0, s>>>(R, P, n4);
    return cudaGetLastError();
}

}  // namespace ecris
