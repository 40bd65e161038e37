// Ion-ion Coulomb collisions of the ECRIS model (arXiv:1507.03392, Sec. II
// collision block): Takizawa-Abe pairing of the ions of each cell and Nanbu's
// scattering angle, Coulomb logarithm lnL_ii.
//
// Per step, after the fused step kernel has given every ion that stayed inside
// its cell (ckey) and its arrival rank in that cell (crank, from an atomic on
// ccount):
//   1. scan      exclusive scan of ccount -> coff (three small passes); the
//                last pass clears ccount and lists the cells holding >= 2 ions;
//   2. scatter   key = (pairing hash << 32 | pid) stored at coff[cell] + rank;
//                the hash is word 0 of the particle's stream-1 Philox block;
//   3. collide   one warp per listed cell sorts its keys (bitonic network in
//                registers, shared memory or global memory by size), so the
//                pairing is independent of the atomic arrival order, then
//                collides consecutive pairs; an odd count puts the first three
//                in a triplet that collides (0,1), (1,2), (2,0) over dt/2 each.
// A collision of ions a, b (same mass M, charges Qa, Qb) over time dt_c uses
//   s = lnL/(4 pi) (Qa Qb e^2 / (eps0 mu))^2 n g^-3 dt_c,  mu = M/2,
// n = w m / V_cell for the cell's m ions; A(s) from coth A - 1/A = e^-s
// (tabulated in FP64 on the host, s >= 1e-3; 1/(1 - e^-s) below, where coth A
// is 1 to working precision; isotropic for s > 6);
//   cos chi = 1 + ln(U + (1-U) e^-2A) / A,  eps = 2 pi U';
// the relative velocity g is turned by (chi, eps) and the change is shared
// equally, which conserves momentum and energy of the pair.
#include "ecris_internal.cuh"

namespace ecris {

namespace {

constexpr int kCollideThreads = 128;
constexpr int kCollideWarps = kCollideThreads / 32;
constexpr int kSmemKeys = 512;    // keys per warp sorted in shared memory (>= 64)

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// pass A: block-local exclusive scan of ccount into coff, block totals to cblk
__global__ void __launch_bounds__(kScanThreads) k_scan_a(const __grid_constant__ RunDev R, uint32_t ncells)
{
    __shared__ uint32_t wsum[kScanThreads / 32];
    const uint32_t base = blockIdx.x * kScanBlock + threadIdx.x * kScanPerThread;
    uint32_t v[kScanPerThread];
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < kScanPerThread; ++j) {
        const uint32_t idx = base + j;
        v[j] = idx < ncells ? R.ccount[idx] : 0u;
        sum += v[j];
    }
    const uint32_t incl = warp_incl_scan(sum);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kScanThreads / 32 ? wsum[lane] : 0u;
        const uint32_t wi = warp_incl_scan(w);
        if (lane < kScanThreads / 32) wsum[lane] = wi - w;
        if (lane == kScanThreads / 32 - 1) R.cblk[blockIdx.x] = wi;
    }
    __syncthreads();
    uint32_t run_off = wsum[warp] + incl - sum;
#pragma unroll
    for (int j = 0; j < kScanPerThread; ++j) {
        const uint32_t idx = base + j;
        if (idx < ncells) R.coff[idx] = run_off;
        run_off += v[j];
    }
}

// pass B: one block scans the block totals in place; coff[ncells] = total
__global__ void __launch_bounds__(1024) k_scan_b(const __grid_constant__ RunDev R, uint32_t nblocks,
                                                 uint32_t ncells)
{
    __shared__ uint32_t wsum[32];
    const uint32_t per = (nblocks + 1023) / 1024;
    const uint32_t base = threadIdx.x * per;
    uint32_t sum = 0;
    for (uint32_t j = 0; j < per; ++j)
        if (base + j < nblocks) sum += R.cblk[base + j];
    const uint32_t incl = warp_incl_scan(sum);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = wsum[lane];
        const uint32_t wi = warp_incl_scan(w);
        wsum[lane] = wi - w;
        if (lane == 31) {
            R.coff[ncells] = wi;
            *R.occ_n = 0u;
        }
    }
    __syncthreads();
    uint32_t off = wsum[warp] + incl - sum;
    for (uint32_t j = 0; j < per; ++j) {
        if (base + j < nblocks) {
            const uint32_t t = R.cblk[base + j];
            R.cblk[base + j] = off;
            off += t;
        }
    }
}

// pass C: add block offsets, clear the counts, list cells with >= 2 ions
__global__ void __launch_bounds__(kScanThreads) k_scan_c(const __grid_constant__ RunDev R, uint32_t ncells)
{
    const uint32_t add = R.cblk[blockIdx.x];
    const uint32_t base = blockIdx.x * kScanBlock;
    for (uint32_t j = threadIdx.x; j < (uint32_t)kScanBlock; j += kScanThreads) {
        const uint32_t idx = base + j;
        if (idx >= ncells) break;
        const uint32_t c = R.ccount[idx];
        if (c) {
            R.ccount[idx] = 0u;
            if (c >= 2u) R.occ[atomicAdd(R.occ_n, 1u)] = idx;
        }
        R.coff[idx] += add;
    }
}

// scatter the pairing keys of the participants into their cell's segment
__global__ void k_scatter(const __grid_constant__ RunDev R, uint32_t n4)
{
    const uint32_t step = *R.step;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n4; g += gridDim.x * blockDim.x) {
        const uint4 k4 = reinterpret_cast<const uint4*>(R.ckey)[g];
        const uint32_t cells[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (cells[j] == kNoCell) continue;
            const uint32_t pid = 4u * g + j;
            const uint32_t slot = R.coff[cells[j]] + R.crank[pid];
            const Words w = rng_words(R, pid, step, 1u);
            R.ckeys[slot] = ((unsigned long long)w.w0 << 32) | pid;
        }
    }
}

// A(s) for 1e-3 <= s <= 6 from the table of ln A, linear in ln s
__device__ __forceinline__ float nanbu_A(const RunDev& R, float s)
{
    if (s < (float)kNanbuSLo) return 1.0f / (-expm1f(-s));
    float t = (logf(s) - R.nanbu_lnlo) * R.nanbu_inv_dln;
    t = fminf(fmaxf(t, 0.0f), (float)(kNanbuN - 1));
    int i = (int)t;
    if (i > kNanbuN - 2) i = kNanbuN - 2;
    const float f = t - (float)i;
    const float la = (1.0f - f) * __ldg(R.nanbu + i) + f * __ldg(R.nanbu + i + 1);
    return expf(la);
}

__device__ void collide(const RunDev& R, uint32_t a, uint32_t b, float dtc, float m_cell, uint32_t first,
                        uint32_t step)
{
    float vax = R.vx[a], vay = R.vy[a], vaz = R.vz[a];
    float vbx = R.vx[b], vby = R.vy[b], vbz = R.vz[b];
    const uint32_t ma = R.meta[a], mb = R.meta[b];
    R.meta[a] = ma | kEvCoulomb;
    R.meta[b] = mb | kEvCoulomb;
    const float gx = vax - vbx, gy = vay - vby, gz = vaz - vbz;
    const float g2 = gx * gx + gy * gy + gz * gz;
    if (!(g2 > 0.0f)) return;
    const float g = sqrtf(g2);
    const float qq = (float)((ma & kQMask) * (mb & kQMask));
    const float s = R.lnl_ii_coef * (qq * qq) * m_cell * dtc / (g2 * g);
    const Words w = rng_words(R, first, step, 1u);
    const float U = unit01(w.w1);
    float cchi;
    if (!(s <= (float)kNanbuSHi)) {
        cchi = 2.0f * U - 1.0f;
    } else {
        const float A = nanbu_A(R, s);
        cchi = 1.0f + log1pf((1.0f - U) * expm1f(-2.0f * A)) / A;
        cchi = fminf(fmaxf(cchi, -1.0f), 1.0f);
    }
    const float schi = sqrtf(fmaxf(0.0f, 1.0f - cchi * cchi));
    float se, ce;
    sincospif(2.0f * unit01(w.w2), &se, &ce);
    const float gp = sqrtf(gy * gy + gz * gz);
    float hx, hy, hz;
    if (gp > 0.0f) {
        hx = gp * ce;
        hy = -(gx * gy * ce + g * gz * se) / gp;
        hz = -(gx * gz * ce - g * gy * se) / gp;
    } else {
        hx = 0.0f;
        hy = g * ce;
        hz = g * se;
    }
    const float dgx = 0.5f * (gx * (cchi - 1.0f) + hx * schi);
    const float dgy = 0.5f * (gy * (cchi - 1.0f) + hy * schi);
    const float dgz = 0.5f * (gz * (cchi - 1.0f) + hz * schi);
    R.vx[a] = vax + dgx; R.vy[a] = vay + dgy; R.vz[a] = vaz + dgz;
    R.vx[b] = vbx - dgx; R.vy[b] = vby - dgy; R.vz[b] = vbz - dgz;
}

// ascending bitonic sort of buf[0, m) by one warp; every compare-exchange moves
// the smaller key to the lower index, so positions >= m act as +infinity and
// their exchanges are skipped.  Sub-network sizes are powers of two, so block
// and offset come from shifts and masks.
__device__ void warp_bitonic(unsigned long long* buf, uint32_t m)
{
    const int lane = threadIdx.x & 31;
    uint32_t P = 1, lp = 0;
    while (P < m) { P <<= 1; ++lp; }
    for (uint32_t lk = 1; lk <= lp; ++lk) {
        const uint32_t k = 1u << lk;
        for (int lj = (int)lk - 1; lj >= 0; --lj) {
            const uint32_t j = 1u << lj;
            for (uint32_t t = lane; t < P / 2; t += 32) {
                const uint32_t blk = t >> lj, off = t & (j - 1);
                uint32_t lo, hi;
                if (lj == (int)lk - 1) {        // first sub-step: mirrored pairs
                    lo = (blk << lk) + off;
                    hi = (blk << lk) + k - 1 - off;
                } else {                        // half-cleaner
                    lo = (blk << (lj + 1)) + off;
                    hi = lo + j;
                }
                if (hi < m) {
                    const unsigned long long x = buf[lo], y = buf[hi];
                    if (y < x) { buf[lo] = y; buf[hi] = x; }
                }
            }
            __syncwarp();
        }
    }
}

// the same network on 32 keys held one per lane
__device__ __forceinline__ unsigned long long lane_sort32(unsigned long long k, int lane)
{
#pragma unroll
    for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            const int partner = (j == (kk >> 1)) ? (lane ^ (kk - 1)) : (lane ^ j);
            const unsigned long long o = __shfl_sync(0xFFFFFFFFu, k, partner);
            k = (lane < partner) ? (o < k ? o : k) : (o > k ? o : k);
        }
    }
    return k;
}

// half-cleaners j = 16 .. 1 on 32 keys held one per lane
__device__ __forceinline__ unsigned long long lane_clean32(unsigned long long k, int lane)
{
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        const int partner = lane ^ j;
        const unsigned long long o = __shfl_sync(0xFFFFFFFFu, k, partner);
        k = (lane < partner) ? (o < k ? o : k) : (o > k ? o : k);
    }
    return k;
}

__global__ void __launch_bounds__(kCollideThreads, 8) k_collide(const __grid_constant__ RunDev R,
                                                             unsigned int* ticket)
{
    __shared__ unsigned long long sk[kCollideWarps][kSmemKeys];
    __shared__ int s_last;
    const uint32_t step = *R.step;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t nocc = *R.occ_n;
    const uint32_t wstride = gridDim.x * kCollideWarps;
    unsigned long long ncoll = 0;
    const float dt = R.dt;
    for (uint32_t i = blockIdx.x * kCollideWarps + wib; i < nocc; i += wstride) {
        const uint32_t cell = R.occ[i];
        const uint32_t off = R.coff[cell];
        const uint32_t m = R.coff[cell + 1] - off;
        unsigned long long* keys = R.ckeys + off;
        unsigned long long* buf;
        if (m <= 64u) {
            // registers: keys lane and lane + 32; each half is sorted by the
            // 32-lane network, then one mirrored exchange across the halves and
            // half-cleaners finish the 64-key network
            unsigned long long k0 = lane < (int)m ? keys[lane] : ~0ull;
            unsigned long long k1 = lane + 32 < (int)m ? keys[lane + 32] : ~0ull;
            k0 = lane_sort32(k0, lane);
            k1 = lane_sort32(k1, lane);
            if (m > 32u) {
                const unsigned long long o0 = __shfl_sync(0xFFFFFFFFu, k1, 31 - lane);
                const unsigned long long o1 = __shfl_sync(0xFFFFFFFFu, k0, 31 - lane);
                k0 = o0 < k0 ? o0 : k0;
                k1 = o1 > k1 ? o1 : k1;
                k0 = lane_clean32(k0, lane);
                k1 = lane_clean32(k1, lane);
            }
            buf = sk[wib];
            buf[lane] = k0;
            buf[lane + 32] = k1;
            __syncwarp();
        } else if (m <= (uint32_t)kSmemKeys) {
            buf = sk[wib];
            for (uint32_t t = lane; t < m; t += 32) buf[t] = keys[t];
            __syncwarp();
            warp_bitonic(buf, m);
        } else {
            buf = keys;   // large cell: sort in place in global memory
            warp_bitonic(buf, m);
        }
        const float mc = (float)m;
        uint32_t start = 0;
        if (m & 1u) {
            if (lane == 0) {
                const uint32_t p0 = (uint32_t)buf[0], p1 = (uint32_t)buf[1], p2 = (uint32_t)buf[2];
                collide(R, p0, p1, 0.5f * dt, mc, p0, step);
                collide(R, p1, p2, 0.5f * dt, mc, p1, step);
                collide(R, p2, p0, 0.5f * dt, mc, p2, step);
            }
            start = 3;
            __syncwarp();
        }
        const uint32_t npairs = (m - start) / 2;
        for (uint32_t p = lane; p < npairs; p += 32) {
            const uint32_t a = (uint32_t)buf[start + 2 * p], b = (uint32_t)buf[start + 2 * p + 1];
            collide(R, a, b, dt, mc, a, step);
        }
        if (lane == 0) ncoll += npairs + (start ? 3u : 0u);
        __syncwarp();
    }
    if (lane == 0 && ncoll) atomicAdd(R.tally + kTallyCoulomb, ncoll);
    // the last block to finish advances the run's step counter
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int prev = atomicAdd(ticket, 1u);
        s_last = (prev == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        *R.step += 1u;
        *ticket = 0u;
    }
}

}  // namespace

int coulomb_scan_blocks(uint32_t ncells) { return (int)((ncells + kScanBlock - 1) / kScanBlock); }

int collide_blocks_per_sm()
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_collide, kCollideThreads, 0) != cudaSuccess || b < 1)
        b = 1;
    return b;
}

cudaError_t launch_coulomb(const RunDev& R, uint32_t ncells, uint32_t n4, unsigned int* ticket, int grid,
                           cudaStream_t s)
{
    const int nb = coulomb_scan_blocks(ncells);
    k_scan_a<<<nb, kScanThreads, 0, s>>>(R, ncells);
    k_scan_b<<<1, 1024, 0, s>>>(R, (uint32_t)nb, ncells);
    k_scan_c<<<nb, kScanThreads, 0, s>>>(R, ncells);
    int sb = (int)((n4 + 255) / 256);
    if (sb > 8192) sb = 8192;
    if (sb < 1) sb = 1;
    k_scatter<<<sb, 256, 0, s>>>(R, n4);
    k_collide<<<grid, kCollideThreads, 0, s>>>(R, ticket);
    return cudaGetLastError();
}

}  // namespace ecris
