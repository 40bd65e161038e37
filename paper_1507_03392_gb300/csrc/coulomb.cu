// Ion-ion Coulomb collisions of the ECRIS model (arXiv:1507.03392, Sec. II
// collision block): Takizawa-Abe pairing of the ions of each cell and Nanbu's
// scattering angle, Coulomb logarithm lnL_ii.
//
// Per step, after the fused step kernel has counted the ions that stayed inside
// per cell (ccount) and published each one's (pid, cell) and (v, Q) record in
// its tile's participant list:
//   1. scan      exclusive scan of ccount -> coff (one pass, decoupled look-back;
//                the kernel lives in step_kernel.cu beside the leaver pass it
//                can run in extra blocks);
//   2. scatter   each participant takes slot coff[cell] + (ccount[cell] counted
//                down by one), which leaves ccount at zero for the next step;
//                the slot receives key = (pairing hash << 32 | pid), the hash
//                being word 0 of the particle's stream-1 Philox block, and the
//                record (v, cell << 6 | Q), so each cell's records are contiguous;
//   3. cells     each block takes the cells whose segments start in its
//                range of participants (kCellIons at the first step after a
//                load; later as many as keep the largest cell of the step
//                before inside shared memory) and copies their keys,
//                records and array slots to shared memory; one thread per
//                participant counts the hashes of its cell that are smaller
//                than its own, which is its place in the cell's order (by hash,
//                then pid: a tie of hash words, about one pair in 2^32, sends
//                the range to a count by the whole key), independent of the
//                atomic arrival order.  Consecutive
//                ranks pair up; a cell with an odd count puts ranks 0, 1, 2 in a
//                triplet that collides (0,1), (1,2), (2,0) over dt/2 each.  The
//                first ion of every pair and triplet is listed in shared memory
//                and one thread per listed entry collides it and writes the
//                velocities back.  A range too large for shared memory (a cell
//                with thousands of ions) is done the same way in global memory.
// A collision of ions a, b (same mass M, charges Qa, Qb) over time dt_c uses
//   s = lnL/(4 pi) (Qa Qb e^2 / (eps0 mu))^2 n g^-3 dt_c,  mu = M/2,
// n = w m / V_cell for the cell's m ions; A(s) from coth A - 1/A = e^-s
// (tabulated in FP64 on the host, s >= 1e-3; 1/(1 - e^-s) below, where coth A
// is 1 to working precision; isotropic for s > 6);
//   cos chi = 1 + ln(U + (1-U) e^-2A) / A,  eps = 2 pi U'
// (the logarithm's argument formed without cancellation in FP32, see collide_w);
// the relative velocity g is turned by (chi, eps) and the change is shared
// equally, which conserves momentum and energy of the pair.
#include "ecris_internal.cuh"

namespace ecris {

namespace {


// scatter the participants of each tile into their cells' segments; counting
// ccount back down gives each its slot and leaves ccount zero for the next step.
// Neighbouring list entries mostly share a cell (the step kernel sees the
// particles sorted by cell), so each run of equal cells within a warp takes
// its slots with one atomic.
__global__ void k_scatter(const __grid_constant__ RunDev R, uint32_t ntiles)
{
    pdl_wait();
    const uint32_t step = *R.step;
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint32_t np = R.tcount[t];
        const uint32_t end = (np + 31u) & ~31u;   // whole warps iterate together
        for (uint32_t i = threadIdx.x; i < end; i += blockDim.x) {
            const bool in = i < np;
            uint4 pc = make_uint4(0u, kNoCell, 0u, 0u);   // (array slot, cell, id, -)
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (in) {
                pc = R.plist[t * R.tile + i];
                v = R.pvel[t * R.tile + i];
            }
            const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, pc.y, 1);
            const uint32_t heads = __ballot_sync(0xFFFFFFFFu, lane == 0 || prev != pc.y);
            const uint32_t upto = 0xFFFFFFFFu >> (31u - lane);             // lanes 0..lane
            const uint32_t after = heads & ~upto;                           // run heads above this lane
            const uint32_t tl = after ? (uint32_t)(__ffs(after) - 2) : 31u; // last lane of this lane's run
            const uint32_t h = 31u - (uint32_t)__clz(heads & upto);          // first lane of this lane's run
            uint32_t top = 0;
            if (in && lane == tl) top = atomicSub(R.ccount + pc.y, tl - h + 1u);
            top = __shfl_sync(0xFFFFFFFFu, top, tl);
            if (!in) continue;
            const uint32_t slot = R.coff[pc.y] + top - 1u - (tl - lane);
            const Words w = rng_words(R, pc.z, step, 1u);
            R.ckeys[slot] = ((unsigned long long)w.w0 << 32) | pc.z;
            R.crec[slot] = make_float4(v.x, v.y, v.z, __uint_as_float((pc.y << 6) | __float_as_uint(v.w)));
            R.cslot[slot] = pc.x;
        }
    }
}

// A(s) for 1e-3 <= s <= 6 from the table of ln A, linear in ln s.  The
// logarithm that indexes the table and the exponential of the interpolated
// ln A use the fast intrinsics: their errors (below 1e-6 in ln s and a few
// units in the last place of A) move A by far less than the table's own
// interpolation error.
__device__ __forceinline__ float nanbu_A(const RunDev& R, float s)
{
    if (s < (float)kNanbuSLo) return 1.0f / (-expm1f(-s));
    float t = (__logf(s) - R.nanbu_lnlo) * R.nanbu_inv_dln;
    t = fminf(fmaxf(t, 0.0f), (float)(kNanbuN - 1));
    int i = (int)t;
    if (i > kNanbuN - 2) i = kNanbuN - 2;
    const float f = t - (float)i;
    const float a0 = __ldg(R.nanbu + i);
    const float la = fmaf(f, __ldg(R.nanbu + i + 1) - a0, a0);
    return __expf(la);
}

// One collision over time dtc of the records ra, rb (vx, vy, vz, Q bits),
// with w1, w2 the stream-1 words 1 and 2 of the pair's first particle (the
// angles); updates the records in place.
__device__ __forceinline__ void collide_w(const RunDev& R, float4& ra, float4& rb, float dtc, float m_cell,
                                          uint32_t w1, uint32_t w2)
{
    // (FMAs written out: this file is compiled without contraction, so that
    // every inlined copy of this code rounds the same way, whichever path of
    // the collision kernel takes a cell)
    const float gx = ra.x - rb.x, gy = ra.y - rb.y, gz = ra.z - rb.z;
    const float g2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
    if (!(g2 > 0.0f)) return;
    // 1/g through the approximate reciprocal square root (a few units in the
    // last place): it sets s and the scattering geometry, not the angle's
    // small-angle digits (those come from eps below)
    const float rg = rsqrtf(g2);
    const float g = g2 * rg;
    const float qq = (float)((__float_as_uint(ra.w) & 63u) * (__float_as_uint(rb.w) & 63u));
    const float s = R.lnl_ii_coef * (qq * qq) * m_cell * dtc * (rg * rg * rg);
    const float U = unit01(w1);
    // eps = 1 - cos chi and epc = 1 + cos chi, each formed without
    // cancellation: in a small-angle collision cos chi lies within FP32
    // rounding of 1, so sin chi = sqrt(1 - cos^2 chi) would lose most of its
    // digits, while sin chi = sqrt(eps epc) keeps them
    float eps, epc;
    if (!(s <= (float)kNanbuSHi)) {
        eps = 2.0f * (1.0f - U);   // isotropic: cos chi = 2U - 1 (both exact in FP32)
        epc = 2.0f * U;
    } else {
        const float A = nanbu_A(R, s);
        // ln(U + (1-U) e^-2A): for small A the sum is close to 1 and log1p of
        // (1-U)(e^-2A - 1) keeps its precision; for larger A the two positive
        // terms are formed directly, since e^-2A can lie below the FP32
        // spacing of expm1 near -1 while U is small as well
        const float lnarg = A < 0.5f ? log1pf((1.0f - U) * expm1f(-2.0f * A))
                                     : logf(fmaf(1.0f - U, expf(-2.0f * A), U));
        eps = fminf(fmaxf(__fdividef(-lnarg, A), 0.0f), 2.0f);
        epc = 2.0f - eps;
    }
    const float schi = sqrt_approx(eps * epc);
    float se, ce;
    sincos_2pi(unit01(w2), &se, &ce);
    const float gp2 = fmaf(gy, gy, gz * gz);
    float hx, hy, hz;
    if (gp2 > 0.0f) {
        const float rgp = rsqrtf(gp2);
        hx = gp2 * rgp * ce;
        hy = -fmaf(gx * gy, ce, g * gz * se) * rgp;
        hz = -fmaf(gx * gz, ce, -(g * gy * se)) * rgp;
    } else {
        hx = 0.0f;
        hy = g * ce;
        hz = g * se;
    }
    const float dgx = 0.5f * fmaf(hx, schi, -(gx * eps));
    const float dgy = 0.5f * fmaf(hy, schi, -(gy * eps));
    const float dgz = 0.5f * fmaf(hz, schi, -(gz * eps));
    ra.x += dgx; ra.y += dgy; ra.z += dgz;
    rb.x -= dgx; rb.y -= dgy; rb.z -= dgz;
}

// the same with the words of particle `first` at this step
__device__ __forceinline__ void collide(const RunDev& R, float4& ra, float4& rb, float dtc, float m_cell,
                                        uint32_t first, uint32_t step)
{
    const Words w = rng_words(R, first, step, 1u);
    collide_w(R, ra, rb, dtc, m_cell, w.w1, w.w2);
}

__device__ __forceinline__ void write_back(const RunDev& R, uint32_t slot, const float4& r)
{
    R.vx[slot] = r.x;
    R.vy[slot] = r.y;
    R.vz[slot] = r.z;
    atomicOr(R.meta + slot, kEvCoulomb);   // result unused: a fire-and-forget reduction
}

// Shared-memory image of one range of cells (see the header).  The pairing
// key (hash << 32 | pid) is kept as its two words.
struct CellSmem {
    uint32_t hash[kCellCap];
    uint32_t pid[kCellCap];
    float4 rec[kCellCap];
    uint32_t slot[kCellCap];
    uint32_t sidx[kCellCap];          // sorted position -> index in the range
    uint2 start[kCellCap / 2 + 1];    // (sorted position, cell count): pairs from the front,
                                      // triplets from the back, so a warp runs one kind
    uint32_t claim[kCellCap / 32];    // sorted positions taken by the 32-bit ranking
    uint32_t npair, ntrip;
    uint32_t s0, s1;
    int tie;                          // two keys of a cell share their hash word
    unsigned long long ncoll;
};

// collide the pair (kind 0) or triplet (kind 1) starting at sorted position p
// of a range (key / rec / slot indexed through sidx), m ions in the cell
template <class K, class V, class S, class I>
__device__ __forceinline__ uint32_t collide_entry(const RunDev& R, const K& key, const V& rec, const S& slot,
                                                  const I& sidx, uint32_t p, uint32_t m, bool triplet,
                                                  uint32_t step)
{
    const float dt = R.dt;
    const uint32_t ia = sidx[p], ib = sidx[p + 1];
    float4 ra = rec[ia], rb = rec[ib];
    if (!triplet) {
        collide(R, ra, rb, dt, (float)m, (uint32_t)key[ia], step);   // ids give the random words
        write_back(R, slot[ia], ra);
        write_back(R, slot[ib], rb);
        return 1u;
    }
    // ranks 0, 1, 2: (0,1), (1,2), (2,0) over dt/2 each; the three pairs'
    // random words do not depend on the velocities, so they are drawn first
    const uint32_t ic = sidx[p + 2];
    float4 rc = rec[ic];
    const float mc = (float)m;
    const Words wa = rng_words(R, (uint32_t)key[ia], step, 1u);
    const Words wb = rng_words(R, (uint32_t)key[ib], step, 1u);
    const Words wc = rng_words(R, (uint32_t)key[ic], step, 1u);
    collide_w(R, ra, rb, 0.5f * dt, mc, wa.w1, wa.w2);
    collide_w(R, rb, rc, 0.5f * dt, mc, wb.w1, wb.w2);
    collide_w(R, rc, ra, 0.5f * dt, mc, wc.w1, wc.w2);
    write_back(R, slot[ia], ra);
    write_back(R, slot[ib], rb);
    write_back(R, slot[ic], rc);
    return 3u;
}

// rank of participant j (index in the range) within its cell: the number of
// smaller keys among the cell's m; seg = the cell's first index in the range
template <class K>
__device__ __forceinline__ uint32_t rank_in_cell(const K& key, uint32_t seg, uint32_t m, unsigned long long mine)
{
    uint32_t r0 = 0, r1 = 0;
    uint32_t i = 0;
    for (; i + 2 <= m; i += 2) {
        r0 += key[seg + i] < mine ? 1u : 0u;
        r1 += key[seg + i + 1] < mine ? 1u : 0u;
    }
    if (i < m) r0 += key[seg + i] < mine ? 1u : 0u;
    return r0 + r1;
}

// the same from the hash words alone: exact when the cell's hashes are
// distinct (then the order by hash is the order by key); a tie gives two
// participants the same rank, which the caller detects
__device__ __forceinline__ uint32_t rank_in_cell32(const uint32_t* hash, uint32_t seg, uint32_t m, uint32_t mine)
{
    const uint32_t* h = hash + seg;
    uint32_t r0 = 0, r1 = 0, r2 = 0, r3 = 0;
    uint32_t i = 0;
    for (; i + 4 <= m; i += 4) {
        r0 += h[i] < mine ? 1u : 0u;
        r1 += h[i + 1] < mine ? 1u : 0u;
        r2 += h[i + 2] < mine ? 1u : 0u;
        r3 += h[i + 3] < mine ? 1u : 0u;
    }
    for (; i < m; ++i) r0 += h[i] < mine ? 1u : 0u;
    return (r0 + r1) + (r2 + r3);
}

// the rank by the whole key (hash, then pid) from the two word arrays
__device__ __forceinline__ uint32_t rank_in_cell64(const uint32_t* hash, const uint32_t* pid, uint32_t seg,
                                                   uint32_t m, uint32_t mh, uint32_t mp)
{
    uint32_t r = 0;
    for (uint32_t i = 0; i < m; ++i) {
        const uint32_t h = hash[seg + i];
        r += (h < mh || (h == mh && pid[seg + i] < mp)) ? 1u : 0u;
    }
    return r;
}

// kind of sorted place r in a cell of m: 1 starts a pair, 2 starts a triplet
__device__ __forceinline__ uint32_t start_kind(uint32_t r, uint32_t m)
{
    if (m < 2u) return 0u;
    if (m & 1u) {
        if (r == 0u) return 2u;
        return (r >= 3u && !((r - 3u) & 1u)) ? 1u : 0u;
    }
    return (r & 1u) ? 0u : 1u;
}

__global__ void __launch_bounds__(256, 6) k_cells(const __grid_constant__ RunDev R, uint32_t ncells, unsigned int* ticket)
{
    extern __shared__ __align__(16) unsigned char cell_smem_raw[];
    CellSmem& S = *reinterpret_cast<CellSmem*>(cell_smem_raw);
    pdl_wait();
    const uint32_t total = R.coff[ncells];
    const uint32_t step = *R.step;
    const uint32_t tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) S.ncoll = 0ull;
    uint32_t ncoll = 0;
    const uint32_t stride = R.crange[0];   // participants a range, as the scan marked them
    for (uint32_t b = blockIdx.x; b * stride < total; b += gridDim.x) {
        if (tid == 0) {
            const uint32_t hi = (b + 1u) * stride;
            S.s0 = R.cstart[b];
            S.s1 = hi >= total ? total : R.cstart[b + 1];
            S.npair = 0u;
            S.ntrip = 0u;
        }
        __syncthreads();
        const uint32_t s0 = S.s0, n = S.s1 - S.s0;
        if (n <= (uint32_t)kCellCap) {
            for (uint32_t j = tid; j < n; j += blockDim.x) {
                const unsigned long long k = R.ckeys[s0 + j];
                S.hash[j] = (uint32_t)(k >> 32);
                S.pid[j] = (uint32_t)k;
                S.rec[j] = R.crec[s0 + j];
                S.slot[j] = R.cslot[s0 + j];
            }
            for (uint32_t w = tid; w < kCellCap / 32; w += blockDim.x) S.claim[w] = 0u;
            if (tid == 0) S.tie = 0;
            __syncthreads();
            // ranks, and the list of pair / triplet starters.  First by the
            // hash words alone, each participant claiming its sorted place;
            // if two claim one place (hash words tie, about once in 2^32
            // pairs), again by the whole key.
            const uint32_t end = (n + 31u) & ~31u;
            for (int exact = 0; exact < 2; ++exact) {
                for (uint32_t j = tid; j < end; j += blockDim.x) {
                    uint32_t kind = 0u, pos = 0u, m = 0u;
                    if (j < n) {
                        const uint32_t cell = __float_as_uint(S.rec[j].w) >> 6;
                        const uint32_t seg = R.coff[cell] - s0;
                        m = R.coff[cell + 1] - R.coff[cell];
                        uint32_t r;
                        if (!exact) {
                            r = rank_in_cell32(S.hash, seg, m, S.hash[j]);
                            const uint32_t bit = 1u << ((seg + r) & 31u);
                            if (atomicOr(&S.claim[(seg + r) >> 5], bit) & bit) S.tie = 1;
                        } else {
                            r = rank_in_cell64(S.hash, S.pid, seg, m, S.hash[j], S.pid[j]);
                        }
                        pos = seg + r;
                        S.sidx[pos] = j;
                        kind = start_kind(r, m);
                    }
                    const uint32_t b1 = __ballot_sync(0xFFFFFFFFu, kind == 1u);
                    const uint32_t b2 = __ballot_sync(0xFFFFFFFFu, kind == 2u);
                    if (b1 | b2) {
                        uint32_t base1 = 0, base2 = 0;
                        if (lane == 0) {
                            if (b1) base1 = atomicAdd(&S.npair, (uint32_t)__popc(b1));
                            if (b2) base2 = atomicAdd(&S.ntrip, (uint32_t)__popc(b2));
                        }
                        base1 = __shfl_sync(0xFFFFFFFFu, base1, 0);
                        base2 = __shfl_sync(0xFFFFFFFFu, base2, 0);
                        const uint32_t below = (1u << lane) - 1u;
                        if (kind == 1u) S.start[base1 + (uint32_t)__popc(b1 & below)] = make_uint2(pos, m);
                        if (kind == 2u)
                            S.start[kCellCap / 2 - (base2 + (uint32_t)__popc(b2 & below))] = make_uint2(pos, m);
                    }
                }
                __syncthreads();
                if (exact || !S.tie) break;
                // a tie: rebuild the lists by the whole key
                if (tid == 0) {
                    S.npair = 0u;
                    S.ntrip = 0u;
                }
                __syncthreads();
            }
            // triplets (three collisions in a row) first, so that they run
            // beside the pairs instead of after them
            const uint32_t np = S.npair, nt = S.ntrip;
            for (uint32_t e = tid; e < nt + np; e += blockDim.x) {
                const bool trip = e < nt;
                const uint2 st = S.start[trip ? kCellCap / 2 - e : e - nt];
                ncoll += collide_entry(R, S.pid, S.rec, S.slot, S.sidx, st.x, st.y, trip, step);
            }
        } else {
            // the same in global memory: sorted positions in sslot
            const unsigned long long* key = R.ckeys + s0;
            const float4* rec = R.crec + s0;
            const uint32_t* slot = R.cslot + s0;
            uint32_t* sidx = R.sslot + s0;
            for (uint32_t j = tid; j < n; j += blockDim.x) {
                const uint32_t cell = __float_as_uint(rec[j].w) >> 6;
                const uint32_t seg = R.coff[cell] - s0;
                const uint32_t m = R.coff[cell + 1] - R.coff[cell];
                sidx[seg + rank_in_cell(key, seg, m, key[j])] = j;
            }
            __syncthreads();
            for (uint32_t p = tid; p < n; p += blockDim.x) {
                const uint32_t cell = __float_as_uint(rec[sidx[p]].w) >> 6;
                const uint32_t seg = R.coff[cell] - s0;
                const uint32_t m = R.coff[cell + 1] - R.coff[cell];
                const uint32_t kind = start_kind(p - seg, m);
                if (kind) ncoll += collide_entry(R, key, rec, slot, sidx, p, m, kind == 2u, step);
            }
        }
        __syncthreads();   // the range's shared memory is reused by the next one
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ncoll += __shfl_down_sync(0xFFFFFFFFu, ncoll, o);
    if (lane == 0 && ncoll) atomicAdd(&S.ncoll, (unsigned long long)ncoll);
    __shared__ int s_last;
    __syncthreads();
    if (tid == 0) {
        if (S.ncoll) atomicAdd(R.tally + kTallyCoulomb, S.ncoll);
        // the last block to finish advances the run's step counter
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1 ? 1 : 0;
    }
    __syncthreads();
    if (s_last && tid == 0) {
        *R.step += 1u;
        *ticket = 0u;
        if (R.nleave) *R.nleave = 0u;   // the leaver pass of the step (if the scan did it) is over
        // the next step's range size: as large as keeps this step's largest
        // cell, with a range's cells whole, inside shared memory
        const uint32_t mx = R.crange[1];
        const uint32_t room = mx < (uint32_t)kCellCap ? (uint32_t)kCellCap - mx : 0u;
        R.crange[0] = min(max(room, (uint32_t)kCellIonsMin), (uint32_t)kCellIonsMax);
        R.crange[1] = 0u;
    }
}

}  // namespace

int coulomb_scan_blocks(uint32_t ncells) { return (int)((ncells + kScanBlock - 1) / kScanBlock); }

int collide_blocks_per_sm()
{
    const int smem = (int)sizeof(CellSmem);
    if (cudaFuncSetAttribute(k_cells, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_cells, 256, smem) != cudaSuccess || b < 1) b = 1;
    return b;
}

// the scatter's grid: at most 32 blocks an SM, each taking tiles b, b + grid, ...
// (fewer, longer-lived blocks than one a tile took 1.4 us less a step at 4e6
// particles)
static uint32_t scatter_grid(uint32_t ntiles)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return ntiles;
    return min(ntiles, 32u * (uint32_t)sms);
}

cudaError_t launch_coulomb(const RunDev& R, uint32_t ncells, uint32_t ntiles, unsigned int* ticket, int grid,
                           uint32_t leave_blocks, int do_leave, cudaStream_t s)
{
    const int nb = coulomb_scan_blocks(ncells);
    cudaError_t e = launch_scan(R, ncells, (uint32_t)nb, leave_blocks, do_leave, s);
    if (e == cudaSuccess && ntiles > 0) e = launch_pdl(k_scatter, dim3(scatter_grid(ntiles)), dim3(256), 0, s, R, ntiles);
    if (e == cudaSuccess) e = launch_pdl(k_cells, dim3(grid), dim3(256), sizeof(CellSmem), s, R, ncells, ticket);
    return e;
}

}  // namespace ecris
