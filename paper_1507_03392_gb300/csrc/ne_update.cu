// Self-consistent electron density on the device (Sec. II: by charge
// neutrality n_e equals the ion charge density), and the atom gate the step
// kernel derives from the largest n_e of each zone.
//
// An update runs in stream order after the steps it averages, with no read
// back to the host:
//   1. n_e of every cell = w (charge now - charge at the mark) / (steps V_cell),
//      in FP64; the mark moves to the charge now; the largest FP32 n_e of the
//      cold and the warm cells is kept;
//   2. every cell's record {n_e, zone, delta_x, delta_y} is rebuilt from
//      those densities: delta follows the printed 3x3 stencil (y-differences
//      for delta_x, x-differences for delta_y, neighbours outside the mesh
//      take the edge value) times -R_L / n_e, R_L = 2.38e-6 sqrt(T_e)/(B dX)
//      (the heating kick of Sec. II), and delta = 0 where n_e = 0 or under
//      isotropic heating;
//   3. the atom gate: the FP32 product n_e k_0 dt, largest over the cells,
//      with a relative margin of 1e-4, turned into the ionisation word
//      ceil((1 - exp(-lambda)) 2^32) above which no cell can ionise an atom.
// This file is compiled without contraction of multiplies and adds, so the
// FP64 arithmetic rounds as the host's own construction of the records does.
#include <cstdint>

#include "ecris_internal.cuh"

namespace ecris {

namespace {

__global__ void k_ne_cells(const unsigned long long* __restrict__ charge, unsigned long long* __restrict__ mark,
                           double* __restrict__ ne, const float4* __restrict__ cell, uint32_t ncells,
                           double weight, double steps_vol, uint32_t* __restrict__ zone_max)
{
    uint32_t m0 = 0u, m1 = 0u;   // FP32 bits of the largest n_e (non-negative: bits order as values)
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
        const unsigned long long q = charge[c];
        const double v = weight * (double)(q - mark[c]) / steps_vol;
        ne[c] = v;
        mark[c] = q;
        const uint32_t b = __float_as_uint((float)v);
        if (cell[c].y > 0.5f) m1 = max(m1, b);
        else m0 = max(m0, b);
    }
    m0 = __reduce_max_sync(0xFFFFFFFFu, m0);
    m1 = __reduce_max_sync(0xFFFFFFFFu, m1);
    if ((threadIdx.x & 31) == 0) {
        if (m0) atomicMax(zone_max, m0);
        if (m1) atomicMax(zone_max + 1, m1);
    }
}

__global__ void k_ne_delta(const double* __restrict__ ne, const double* __restrict__ rl_coef,
                           float4* __restrict__ cell, int nx, int ny, uint32_t ncells, int isoheat)
{
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
        const int ix = (int)(c % (uint32_t)nx);
        const int iy = (int)((c / (uint32_t)nx) % (uint32_t)ny);
        const uint32_t plane = c - (uint32_t)(iy * nx + ix);   // first cell of the z layer
        auto NE = [&](int jy, int jx) {
            jy = jy < 0 ? 0 : (jy >= ny ? ny - 1 : jy);
            jx = jx < 0 ? 0 : (jx >= nx ? nx - 1 : jx);
            return ne[plane + (uint32_t)(jy * nx + jx)];
        };
        const double v = ne[c];
        double dlx = 0.0, dly = 0.0;
        if (v > 0.0 && !isoheat) {
            const double rl = rl_coef[c] / v;
            const double sx = NE(iy - 1, ix) - NE(iy + 1, ix) +
                              0.5 * (NE(iy - 1, ix + 1) + NE(iy - 1, ix - 1) - NE(iy + 1, ix - 1) - NE(iy + 1, ix + 1));
            const double sy = NE(iy, ix + 1) - NE(iy, ix - 1) +
                              0.5 * (NE(iy + 1, ix + 1) + NE(iy - 1, ix + 1) - NE(iy + 1, ix - 1) - NE(iy - 1, ix - 1));
            dlx = -rl * sx;
            dly = -rl * sy;
        }
        const float zone = cell[c].y;
        cell[c] = make_float4((float)v, zone, (float)dlx, (float)dly);
    }
}

// words: [0] the gate, [1], [2] FP32 bits of the largest n_e of the cold and
// warm cells; kdt: k dt by zone and Q (zone 0 at 0, zone 1 at kQSlots)
__global__ void k_atom_gate(uint32_t* words, const float* kdt)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const float lam = fmaxf(__uint_as_float(words[1]) * kdt[0], __uint_as_float(words[2]) * kdt[kQSlots]);
    const float lam_max = lam * 1.0001f;
    const double pmax = -expm1(-(double)lam_max);
    const double gate = ceil(pmax * 4294967296.0);
    words[0] = gate >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)gate;
}

int grid_for(uint32_t ncells, int sm_count)
{
    const uint32_t want = (ncells + 255u) / 256u;
    const uint32_t cap = (uint32_t)(sm_count > 0 ? sm_count : 1) * 8u;
    return (int)(want < 1u ? 1u : (want > cap ? cap : want));
}

}  // namespace

cudaError_t launch_atom_gate(float* kdt, cudaStream_t s)
{
    k_atom_gate<<<1, 32, 0, s>>>(reinterpret_cast<uint32_t*>(kdt + kGateWord), kdt);
    return cudaGetLastError();
}

cudaError_t launch_ne_update(const unsigned long long* charge, unsigned long long* mark, double* ne,
                             const double* rl_coef, float4* cell, float* kdt, int nx, int ny, uint32_t ncells,
                             double weight, double steps_vol, bool isoheat, int sm_count, cudaStream_t s)
{
    uint32_t* words = reinterpret_cast<uint32_t*>(kdt + kGateWord);
    cudaError_t e = cudaMemsetAsync(words + 1, 0, 2 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const int grid = grid_for(ncells, sm_count);
    k_ne_cells<<<grid, 256, 0, s>>>(charge, mark, ne, cell, ncells, weight, steps_vol, words + 1);
    k_ne_delta<<<grid, 256, 0, s>>>(ne, rl_coef, cell, nx, ny, ncells, isoheat ? 1 : 0);
    k_atom_gate<<<1, 32, 0, s>>>(words, kdt);
    return cudaGetLastError();
}

}  // namespace ecris
