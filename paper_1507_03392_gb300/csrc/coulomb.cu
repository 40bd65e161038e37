// Ion-ion Coulomb collisions of the ECRIS model (arXiv:1507.03392, Sec. II
// collision block): Takizawa-Abe pairing of the ions of each cell and Nanbu's
// scattering angle, Coulomb logarithm lnL_ii.
//
// Per step, after the fused step kernel has counted the ions that stayed inside
// per cell (ccount) and published each one's (pid, cell) and (v, Q) record in
// its tile's participant list:
//   1. scan      exclusive scan of ccount -> coff (three small passes); the
//                last pass lists the cells holding >= 2 ions;
//   2. scatter   each listed participant takes slot coff[cell] + (ccount[cell]
//                counted down by one), which leaves ccount at zero for the next
//                step; the slot receives key = (pairing hash << 32 | pid), the
//                hash being word 0 of the particle's stream-1 Philox block, and
//                the (v, Q) record, so each cell's records become contiguous;
//   3. collide   one warp per listed cell sorts its keys (bitonic network in
//                registers, shared memory or global memory by size), so the
//                pairing is independent of the atomic arrival order, collides
//                consecutive pairs on the contiguous records, and writes the new
//                velocities back; an odd count puts the first three in a
//                triplet that collides (0,1), (1,2), (2,0) over dt/2 each.
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
constexpr int kSmemKeys = 256;    // participants per warp handled in shared memory (>= 64)

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

// pass C: add block offsets, list cells with >= 2 ions
__global__ void __launch_bounds__(kScanThreads) k_scan_c(const __grid_constant__ RunDev R, uint32_t ncells)
{
    const uint32_t add = R.cblk[blockIdx.x];
    const uint32_t base = blockIdx.x * kScanBlock;
    for (uint32_t j = threadIdx.x; j < (uint32_t)kScanBlock; j += kScanThreads) {
        const uint32_t idx = base + j;
        if (idx >= ncells) break;
        if (R.ccount[idx] >= 2u) R.occ[atomicAdd(R.occ_n, 1u)] = idx;
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
            const uint2 pc = R.plist[t * kTile + i];
            const float4 v = R.pvel[t * kTile + i];
            const uint32_t slot = R.coff[pc.y] + atomicSub(R.ccount + pc.y, 1u) - 1u;
            const Words w = rng_words(R, pc.x, step, 1u);
            R.ckeys[slot] = ((unsigned long long)w.w0 << 32) | pc.x;
            R.crec[slot] = v;
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
    const float qq = (float)(__float_as_uint(ra.w) * __float_as_uint(rb.w));
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

__device__ __forceinline__ void write_back(const RunDev& R, uint32_t pid, const float4& r)
{
    R.vx[pid] = r.x;
    R.vy[pid] = r.y;
    R.vz[pid] = r.z;
    atomicOr(R.meta + pid, kEvCoulomb);   // result unused: a fire-and-forget reduction
}

// Ascending bitonic sort of keys[0, m) by one warp, with a payload moved along
// (shared-memory or global arrays).  Every compare-exchange moves the smaller
// key to the lower index, so positions >= m act as +infinity and their
// exchanges are skipped.  Sub-network sizes are powers of two, so block and
// offset come from shifts and masks.
template <class P>
__device__ void warp_bitonic(unsigned long long* keys, P* pay, uint32_t m)
{
    const int lane = threadIdx.x & 31;
    uint32_t P2 = 1, lp = 0;
    while (P2 < m) { P2 <<= 1; ++lp; }
    for (uint32_t lk = 1; lk <= lp; ++lk) {
        const uint32_t k = 1u << lk;
        for (int lj = (int)lk - 1; lj >= 0; --lj) {
            const uint32_t j = 1u << lj;
            for (uint32_t t = lane; t < P2 / 2; t += 32) {
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
                    const unsigned long long x = keys[lo], y = keys[hi];
                    if (y < x) {
                        keys[lo] = y;
                        keys[hi] = x;
                        const P px = pay[lo];
                        pay[lo] = pay[hi];
                        pay[hi] = px;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// one compare-exchange stage across lanes for (key, index) held one per lane
__device__ __forceinline__ void lane_cx(unsigned long long& k, uint32_t& i, int partner, bool low)
{
    const unsigned long long ok = __shfl_sync(0xFFFFFFFFu, k, partner);
    const uint32_t oi = __shfl_sync(0xFFFFFFFFu, i, partner);
    const bool take = low ? (ok < k) : (ok > k);
    if (take) { k = ok; i = oi; }
}

// the bitonic network on 32 (key, index) pairs held one per lane
__device__ __forceinline__ void lane_sort32(unsigned long long& k, uint32_t& i, int lane)
{
#pragma unroll
    for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            const int partner = (j == (kk >> 1)) ? (lane ^ (kk - 1)) : (lane ^ j);
            lane_cx(k, i, partner, lane < partner);
        }
    }
}

// half-cleaners j = 16 .. 1 on 32 pairs held one per lane
__device__ __forceinline__ void lane_clean32(unsigned long long& k, uint32_t& i, int lane)
{
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        const int partner = lane ^ j;
        lane_cx(k, i, partner, lane < partner);
    }
}

__global__ void __launch_bounds__(kCollideThreads, 8) k_collide(const __grid_constant__ RunDev R,
                                                                unsigned int* ticket)
{
    __shared__ unsigned long long sk[kCollideWarps][kSmemKeys];
    __shared__ uint16_t si[kCollideWarps][kSmemKeys];
    __shared__ float4 sr[kCollideWarps][kSmemKeys];
    __shared__ int s_last;
    const uint32_t step = *R.step;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t nocc = *R.occ_n;
    const uint32_t wstride = gridDim.x * kCollideWarps;
    unsigned long long ncoll = 0;
    const float dt = R.dt;
    for (uint32_t c = blockIdx.x * kCollideWarps + wib; c < nocc; c += wstride) {
        const uint32_t cell = R.occ[c];
        const uint32_t off = R.coff[cell];
        const uint32_t m = R.coff[cell + 1] - off;
        unsigned long long* gk = R.ckeys + off;
        float4* gr = R.crec + off;
        const float mc = (float)m;
        const uint32_t start = (m & 1u) ? 3u : 0u;
        const uint32_t npairs = (m - start) / 2;
        if (m <= (uint32_t)kSmemKeys) {
            unsigned long long* K = sk[wib];
            uint16_t* I = si[wib];
            float4* Rc = sr[wib];
            for (uint32_t t = lane; t < m; t += 32) Rc[t] = gr[t];
            if (m <= 64u) {
                // registers: pairs lane and lane + 32; each half is sorted by
                // the 32-lane network, then one mirrored exchange across the
                // halves and half-cleaners finish the 64-key network
                unsigned long long k0 = lane < (int)m ? gk[lane] : ~0ull;
                unsigned long long k1 = lane + 32 < (int)m ? gk[lane + 32] : ~0ull;
                uint32_t i0 = lane, i1 = lane + 32;
                lane_sort32(k0, i0, lane);
                if (m > 32u) {
                    lane_sort32(k1, i1, lane);
                    const unsigned long long o0 = __shfl_sync(0xFFFFFFFFu, k1, 31 - lane);
                    const uint32_t oi0 = __shfl_sync(0xFFFFFFFFu, i1, 31 - lane);
                    const unsigned long long o1 = __shfl_sync(0xFFFFFFFFu, k0, 31 - lane);
                    const uint32_t oi1 = __shfl_sync(0xFFFFFFFFu, i0, 31 - lane);
                    if (o0 < k0) { k0 = o0; i0 = oi0; }
                    if (o1 > k1) { k1 = o1; i1 = oi1; }
                    lane_clean32(k0, i0, lane);
                    lane_clean32(k1, i1, lane);
                }
                K[lane] = k0;
                I[lane] = (uint16_t)i0;
                K[lane + 32] = k1;
                I[lane + 32] = (uint16_t)i1;
                __syncwarp();
            } else {
                for (uint32_t t = lane; t < m; t += 32) {
                    K[t] = gk[t];
                    I[t] = (uint16_t)t;
                }
                __syncwarp();
                warp_bitonic(K, I, m);
            }
            if (start) {
                if (lane == 0) {
                    const uint32_t p0 = (uint32_t)K[0], p1 = (uint32_t)K[1], p2 = (uint32_t)K[2];
                    float4 r0 = Rc[I[0]], r1 = Rc[I[1]], r2 = Rc[I[2]];
                    collide(R, r0, r1, 0.5f * dt, mc, p0, step);
                    collide(R, r1, r2, 0.5f * dt, mc, p1, step);
                    collide(R, r2, r0, 0.5f * dt, mc, p2, step);
                    Rc[I[0]] = r0; Rc[I[1]] = r1; Rc[I[2]] = r2;
                }
                __syncwarp();
            }
            for (uint32_t p = lane; p < npairs; p += 32) {
                const uint32_t a = start + 2 * p, b = a + 1;
                float4 ra = Rc[I[a]], rb = Rc[I[b]];
                collide(R, ra, rb, dt, mc, (uint32_t)K[a], step);
                Rc[I[a]] = ra;
                Rc[I[b]] = rb;
            }
            __syncwarp();
            for (uint32_t t = lane; t < m; t += 32) write_back(R, (uint32_t)K[t], Rc[I[t]]);
        } else {
            // large cell: sort keys and records together in place in global memory
            warp_bitonic(gk, gr, m);
            if (start) {
                if (lane == 0) {
                    float4 r0 = gr[0], r1 = gr[1], r2 = gr[2];
                    collide(R, r0, r1, 0.5f * dt, mc, (uint32_t)gk[0], step);
                    collide(R, r1, r2, 0.5f * dt, mc, (uint32_t)gk[1], step);
                    collide(R, r2, r0, 0.5f * dt, mc, (uint32_t)gk[2], step);
                    gr[0] = r0; gr[1] = r1; gr[2] = r2;
                }
                __syncwarp();
            }
            for (uint32_t p = lane; p < npairs; p += 32) {
                const uint32_t a = start + 2 * p, b = a + 1;
                float4 ra = gr[a], rb = gr[b];
                collide(R, ra, rb, dt, mc, (uint32_t)gk[a], step);
                gr[a] = ra;
                gr[b] = rb;
            }
            __syncwarp();
            for (uint32_t t = lane; t < m; t += 32) write_back(R, (uint32_t)gk[t], gr[t]);
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

cudaError_t launch_coulomb(const RunDev& R, uint32_t ncells, uint32_t ntiles, unsigned int* ticket, int grid,
                           cudaStream_t s)
{
    const int nb = coulomb_scan_blocks(ncells);
    k_scan_a<<<nb, kScanThreads, 0, s>>>(R, ncells);
    k_scan_b<<<1, 1024, 0, s>>>(R, (uint32_t)nb, ncells);
    k_scan_c<<<nb, kScanThreads, 0, s>>>(R, ncells);
    if (ntiles > 0) k_scatter<<<ntiles, 256, 0, s>>>(R, ntiles);
    k_collide<<<grid, kCollideThreads, 0, s>>>(R, ticket);
    return cudaGetLastError();
}

}  // namespace ecris
