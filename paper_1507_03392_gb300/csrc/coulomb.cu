// Ion-ion Coulomb collisions of the ECRIS model (arXiv:1507.03392, Sec. II
// collision block): Takizawa-Abe pairing of the ions of each cell and Nanbu's
// scattering angle, Coulomb logarithm lnL_ii.
//
// Per step, after the fused step kernel has counted the ions that stayed inside
// per cell (ccount) and published each one's (pid, cell) and (v, Q) record in
// its tile's participant list:
//   1. scan      exclusive scan of ccount -> coff (three small passes);
//   2. scatter   each participant takes slot coff[cell] + (ccount[cell] counted
//                down by one), which leaves ccount at zero for the next step;
//                the slot receives key = (pairing hash << 32 | pid), the hash
//                being word 0 of the particle's stream-1 Philox block, and the
//                record (v, cell << 6 | Q), so each cell's records are contiguous;
//   3. rank      one thread per participant counts the keys of its cell that
//                are smaller than its own; that rank is its place in the cell's
//                order (by hash, then pid), independent of the atomic arrival
//                order, and the record moves there;
//                Consecutive ranks pair up; a cell with an odd count puts ranks
//                0, 1, 2 in a triplet that collides (0,1), (1,2), (2,0) over
//                dt/2 each; the first ion of every pair and triplet is listed;
//   4. pairs     one thread per listed pair or triplet collides it and writes
//                the new velocities back.
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
            R.npt[0] = 0u;
            R.npt[1] = 0u;
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

// pass C: add block offsets
__global__ void __launch_bounds__(kScanThreads) k_scan_c(const __grid_constant__ RunDev R, uint32_t ncells)
{
    const uint32_t add = R.cblk[blockIdx.x];
    const uint32_t base = blockIdx.x * kScanBlock;
    for (uint32_t j = threadIdx.x; j < (uint32_t)kScanBlock; j += kScanThreads) {
        const uint32_t idx = base + j;
        if (idx >= ncells) break;
        R.coff[idx] += add;
    }
}

// scatter the participants of each tile into their cells' segments; counting
// ccount back down gives each its slot and leaves ccount zero for the next step
__global__ void k_scatter(const __grid_constant__ RunDev R, uint32_t ntiles)
{
    const uint32_t step = *R.step;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint32_t np = R.tcount[t];
        for (uint32_t i = threadIdx.x; i < np; i += blockDim.x) {
            const uint4 pc = R.plist[t * kTile + i];   // (array slot, cell, id, -)
            const float4 v = R.pvel[t * kTile + i];
            const uint32_t slot = R.coff[pc.y] + atomicSub(R.ccount + pc.y, 1u) - 1u;
            const Words w = rng_words(R, pc.z, step, 1u);
            R.ckeys[slot] = ((unsigned long long)w.w0 << 32) | pc.z;
            R.crec[slot] = make_float4(v.x, v.y, v.z, __uint_as_float((pc.y << 6) | __float_as_uint(v.w)));
            R.cslot[slot] = pc.x;
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

// One collision over time dtc of the records ra, rb (vx, vy, vz, Q bits),
// using the stream-1 words of particle `first`; updates the records in place.
__device__ __forceinline__ void collide(const RunDev& R, float4& ra, float4& rb, float dtc, float m_cell,
                                        uint32_t first, uint32_t step)
{
    const float gx = ra.x - rb.x, gy = ra.y - rb.y, gz = ra.z - rb.z;
    const float g2 = gx * gx + gy * gy + gz * gz;
    if (!(g2 > 0.0f)) return;
    const float g = sqrtf(g2);
    const float qq = (float)((__float_as_uint(ra.w) & 63u) * (__float_as_uint(rb.w) & 63u));
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
    ra.x += dgx; ra.y += dgy; ra.z += dgz;
    rb.x -= dgx; rb.y -= dgy; rb.z -= dgz;
}

__device__ __forceinline__ void write_back(const RunDev& R, uint32_t slot, const float4& r)
{
    R.vx[slot] = r.x;
    R.vy[slot] = r.y;
    R.vz[slot] = r.z;
    atomicOr(R.meta + slot, kEvCoulomb);   // result unused: a fire-and-forget reduction
}

// place each participant at its rank within its cell's order, and list the
// first ion of every pair (and of every triplet) for the collision kernel
__global__ void k_rank(const __grid_constant__ RunDev R, uint32_t ncells)
{
    const uint32_t total = R.coff[ncells];
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t end = (total + 31u) & ~31u;   // whole warps iterate together
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < end; j += gridDim.x * blockDim.x) {
        uint32_t kind = 0, slot = 0, m = 0;      // kind 1: starts a pair, 2: starts a triplet
        if (j < total) {
            const unsigned long long key = R.ckeys[j];
            const float4 rec = R.crec[j];
            const uint32_t cell = __float_as_uint(rec.w) >> 6;
            const uint32_t seg = R.coff[cell];
            m = R.coff[cell + 1] - seg;
            uint32_t rank = 0;
            const unsigned long long* k = R.ckeys + seg;
            for (uint32_t i = 0; i < m; ++i) rank += (k[i] < key) ? 1u : 0u;
            slot = seg + rank;
            R.skeys[slot] = key;
            R.srec[slot] = rec;
            R.sslot[slot] = R.cslot[j];
            if (m >= 2u) {
                const uint32_t start = (m & 1u) ? 3u : 0u;
                if ((m & 1u) && rank == 0u) kind = 2;
                else if (rank >= start && !((rank - start) & 1u)) kind = 1;
            }
        }
        // warp-aggregated appends to the pair and triplet lists; the two
        // counter updates are issued together so their latencies overlap
        const uint32_t b1 = __ballot_sync(0xFFFFFFFFu, kind == 1u);
        const uint32_t b2 = __ballot_sync(0xFFFFFFFFu, kind == 2u);
        if (b1 | b2) {
            uint32_t base1 = 0, base2 = 0;
            if (lane == 0) {
                if (b1) base1 = atomicAdd(R.npt, (uint32_t)__popc(b1));
                if (b2) base2 = atomicAdd(R.npt + 1, (uint32_t)__popc(b2));
            }
            base1 = __shfl_sync(0xFFFFFFFFu, base1, 0);
            base2 = __shfl_sync(0xFFFFFFFFu, base2, 0);
            const uint32_t below = (1u << lane) - 1u;
            if (kind == 1u) R.pairs[base1 + (uint32_t)__popc(b1 & below)] = make_uint2(slot, m);
            if (kind == 2u) R.trips[base2 + (uint32_t)__popc(b2 & below)] = make_uint2(slot, m);
        }
    }
}

// one thread per listed pair or triplet: collide it and write the velocities back
__global__ void k_pairs(const __grid_constant__ RunDev R, uint32_t ncells, unsigned int* ticket)
{
    __shared__ int s_last;
    const uint32_t step = *R.step;
    const uint32_t np = R.npt[0], nt = R.npt[1];
    const float dt = R.dt;
    unsigned long long ncoll = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < np + nt; i += gridDim.x * blockDim.x) {
        if (i < np) {
            const uint2 pr = R.pairs[i];
            const uint32_t t = pr.x;
            float4 ra = R.srec[t], rb = R.srec[t + 1];
            collide(R, ra, rb, dt, (float)pr.y, (uint32_t)R.skeys[t], step);   // ids give the random words
            write_back(R, R.sslot[t], ra);
            write_back(R, R.sslot[t + 1], rb);
            ncoll += 1;
        } else {
            // triplet of ranks 0, 1, 2: (0,1), (1,2), (2,0) over dt/2 each
            const uint2 tr = R.trips[i - np];
            const uint32_t t = tr.x;
            const float mc = (float)tr.y;
            float4 ra = R.srec[t], rb = R.srec[t + 1], rc = R.srec[t + 2];
            const uint32_t pa = (uint32_t)R.skeys[t], pb = (uint32_t)R.skeys[t + 1], pc = (uint32_t)R.skeys[t + 2];
            collide(R, ra, rb, 0.5f * dt, mc, pa, step);
            collide(R, rb, rc, 0.5f * dt, mc, pb, step);
            collide(R, rc, ra, 0.5f * dt, mc, pc, step);
            write_back(R, R.sslot[t], ra);
            write_back(R, R.sslot[t + 1], rb);
            write_back(R, R.sslot[t + 2], rc);
            ncoll += 3;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ncoll += __shfl_down_sync(0xFFFFFFFFu, ncoll, o);
    if ((threadIdx.x & 31) == 0 && ncoll) atomicAdd(R.tally + kTallyCoulomb, ncoll);
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
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pairs, 256, 0) != cudaSuccess || b < 1) b = 1;
    return b;
}

cudaError_t launch_coulomb(const RunDev& R, uint32_t ncells, uint32_t ntiles, unsigned int* ticket, int grid,
                           cudaStream_t s)
{
    const int nb = coulomb_scan_blocks(ncells);
    k_scan_a<<<nb, kScanThreads, 0, s>>>(R, ncells);
    k_scan_b<<<1, 1024, 0, s>>>(R, (uint32_t)nb, ncells);
    k_scan_c<<<nb, kScanThreads, 0, s>>>(R, ncells);
    if (ntiles > 0) k_scatter<<<ntiles, 256, 0, s>>>(R, ntiles);
    k_rank<<<grid, 256, 0, s>>>(R, ncells);
    k_pairs<<<grid, 256, 0, s>>>(R, ncells, ticket);
    return cudaGetLastError();
}

}  // namespace ecris
