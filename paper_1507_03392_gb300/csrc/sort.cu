// Particle layout maintenance: a counting sort of a run's particles by
// (ion/atom, cell), and the export of the state in load order.
//
// The sort is a layout choice, not part of the model: every particle carries
// its stable id (the Philox counter word), and every result of the step is
// independent of where a particle sits in the arrays.  Keeping the particles
// grouped lets a warp's lanes take the same branch (ions and atoms run
// different code), share cell records and field samples in L1, add their
// deposits with one reduction per cell, and keeps a cell's ions close together
// for the collision kernels.
//
// Passes: count keys into a histogram (2 Nc + 1 bins: ions by cell, atoms by
// cell, one bin for frozen and padding slots); exclusive scan; move every
// particle to off[key] + (histogram counted down by one), which leaves the
// histogram zero for the next sort.  Order inside a bin follows the atomics
// and does not matter.  The move writes the destination arrays directly when
// the input is mostly in key order already (every sort but the first after a
// load), since a warp's lanes then land on consecutive places and the eight
// arrays' writes coalesce.  For input in arbitrary order it writes one
// 32-byte record per particle, a full sector for a random destination instead
// of eight partial ones, and a second pass unpacks the records coalesced.
#include "ecris_internal.cuh"

namespace ecris {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortPerThread = 8;
constexpr int kSortScanBlock = kSortThreads * kSortPerThread;

__device__ __forceinline__ uint32_t key_of(const RunDev& R, int32_t x, int32_t y, int32_t z, uint32_t m)
{
    const uint32_t nc = R.ncells;
    if (m & (kStFrozen | kStPad)) return 2u * nc;
    return ((m & kQMask) ? 0u : nc) + ngp_cell(R, x, y, z);
}

__device__ __forceinline__ uint32_t sort_key(const RunDev& R, uint32_t i)
{
    return key_of(R, R.x[i], R.y[i], R.z[i], R.meta[i]);
}

// lanes with equal keys add once per group (input already in order makes
// whole warps share a key)
__global__ void k_sort_count(const __grid_constant__ RunDev R, uint32_t cap, uint32_t* __restrict__ hist)
{
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t end = (cap + 31u) & ~31u;   // whole warps iterate together
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < end; i += stride) {
        const bool in = i < cap;
        const uint32_t key = in ? sort_key(R, i) : 0xFFFFFFFFu;
        const uint32_t act = __ballot_sync(0xFFFFFFFFu, in);
        if (!in) continue;
        const uint32_t grp = __match_any_sync(act, key);
        if ((threadIdx.x & 31) == (uint32_t)(__ffs(grp) - 1)) atomicAdd(hist + key, (uint32_t)__popc(grp));
    }
}

__device__ __forceinline__ uint32_t warp_incl(uint32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// block-local exclusive scan of in[0, n) into out, block totals to blk
__global__ void __launch_bounds__(kSortThreads) k_scan1(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                        uint32_t* __restrict__ blk, uint32_t n)
{
    __shared__ uint32_t ws[kSortThreads / 32];
    const uint32_t base = blockIdx.x * kSortScanBlock + threadIdx.x * kSortPerThread;
    uint32_t v[kSortPerThread], sum = 0;
#pragma unroll
    for (int j = 0; j < kSortPerThread; ++j) {
        v[j] = base + j < n ? in[base + j] : 0u;
        sum += v[j];
    }
    const uint32_t incl = warp_incl(sum);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < kSortThreads / 32 ? ws[lane] : 0u;
        const uint32_t wi = warp_incl(w);
        if (lane < kSortThreads / 32) ws[lane] = wi - w;
        if (lane == kSortThreads / 32 - 1) blk[blockIdx.x] = wi;
    }
    __syncthreads();
    uint32_t o = ws[warp] + incl - sum;
#pragma unroll
    for (int j = 0; j < kSortPerThread; ++j) {
        if (base + j < n) out[base + j] = o;
        o += v[j];
    }
}

// one block: exclusive scan of the block totals in place, total to out[n]
__global__ void __launch_bounds__(1024) k_scan2(uint32_t* __restrict__ blk, uint32_t nb, uint32_t* __restrict__ out,
                                                uint32_t n)
{
    __shared__ uint32_t ws[32];
    const uint32_t per = (nb + 1023) / 1024, base = threadIdx.x * per;
    uint32_t sum = 0;
    for (uint32_t j = 0; j < per; ++j)
        if (base + j < nb) sum += blk[base + j];
    const uint32_t incl = warp_incl(sum);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = ws[lane];
        const uint32_t wi = warp_incl(w);
        ws[lane] = wi - w;
        if (lane == 31) out[n] = wi;
    }
    __syncthreads();
    uint32_t o = ws[warp] + incl - sum;
    for (uint32_t j = 0; j < per; ++j) {
        if (base + j < nb) {
            const uint32_t t = blk[base + j];
            blk[base + j] = o;
            o += t;
        }
    }
}

__global__ void __launch_bounds__(kSortThreads) k_scan3(uint32_t* __restrict__ out, const uint32_t* __restrict__ blk,
                                                        uint32_t n)
{
    const uint32_t add = blk[blockIdx.x], base = blockIdx.x * kSortScanBlock;
    for (uint32_t j = threadIdx.x; j < (uint32_t)kSortScanBlock; j += kSortThreads)
        if (base + j < n) out[base + j] += add;
}

// kRecords: write 32-byte records to aos (unpacked by k_sort_unpack), else
// the destination arrays
template <bool kRecords>
__global__ void k_sort_move(const __grid_constant__ RunDev R, uint32_t cap, ParticleSet dst, uint4* __restrict__ aos,
                            uint32_t* __restrict__ hist, const uint32_t* __restrict__ off)
{
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t end = (cap + 31u) & ~31u;
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < end; i += stride) {
        const bool in = i < cap;
        // the particle's words and its bin's offset are loaded before the
        // atomic below, so their round trips overlap instead of following it
        int32_t x = 0, y = 0, z = 0;
        float vx = 0.0f, vy = 0.0f, vz = 0.0f;
        uint32_t meta = 0u, id = 0u, key = 0xFFFFFFFFu;
        if (in) {
            x = R.x[i];
            y = R.y[i];
            z = R.z[i];
            meta = R.meta[i];
            vx = R.vx[i];
            vy = R.vy[i];
            vz = R.vz[i];
            id = R.id[i];
            key = key_of(R, x, y, z, meta);
        }
        const uint32_t act = __ballot_sync(0xFFFFFFFFu, in);
        if (!in) continue;
        const uint32_t base = off[key];
        // one atomic per group of lanes with the same key; lanes take
        // consecutive places below the group's previous count
        const uint32_t grp = __match_any_sync(act, key);
        const uint32_t leader = (uint32_t)(__ffs(grp) - 1);
        uint32_t top = 0;
        if (lane == leader) top = atomicSub(hist + key, (uint32_t)__popc(grp));
        top = __shfl_sync(grp, top, leader);
        const uint32_t rank = (uint32_t)__popc(grp & ((1u << lane) - 1u));
        const uint32_t d = base + top - 1u - rank;
        if (kRecords) {
            aos[2 * d] = make_uint4((uint32_t)x, (uint32_t)y, (uint32_t)z, __float_as_uint(vx));
            aos[2 * d + 1] = make_uint4(__float_as_uint(vy), __float_as_uint(vz), meta, id);
        } else {
            dst.x[d] = x;
            dst.y[d] = y;
            dst.z[d] = z;
            dst.vx[d] = vx;
            dst.vy[d] = vy;
            dst.vz[d] = vz;
            dst.meta[d] = meta;
            dst.id[d] = id;
        }
    }
}

// records in sorted order -> the destination arrays, coalesced both ways
__global__ void k_sort_unpack(const uint4* __restrict__ aos, uint32_t cap, ParticleSet dst)
{
    for (uint32_t d = blockIdx.x * blockDim.x + threadIdx.x; d < cap; d += gridDim.x * blockDim.x) {
        const uint4 a = aos[2 * d], b = aos[2 * d + 1];
        dst.x[d] = (int32_t)a.x;
        dst.y[d] = (int32_t)a.y;
        dst.z[d] = (int32_t)a.z;
        dst.vx[d] = __uint_as_float(a.w);
        dst.vy[d] = __uint_as_float(b.x);
        dst.vz[d] = __uint_as_float(b.y);
        dst.meta[d] = b.z;
        dst.id[d] = b.w;
    }
}

struct OutPtrs { float* p[6]; };

__global__ void k_export_ordered(const __grid_constant__ RunDev R, uint32_t n, uint32_t cap, OutPtrs out,
                                 uint32_t* __restrict__ meta_out, double sxy, double sz)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
        const uint32_t d = R.id[i];
        if (d >= n) continue;   // padding
        if (out.p[0]) out.p[0][d] = (float)((double)R.x[i] * sxy);
        if (out.p[1]) out.p[1][d] = (float)((double)R.y[i] * sxy);
        if (out.p[2]) out.p[2][d] = (float)(((double)R.z[i] + 2147483648.0) * sz);
        if (out.p[3]) out.p[3][d] = R.vx[i];
        if (out.p[4]) out.p[4][d] = R.vy[i];
        if (out.p[5]) out.p[5][d] = R.vz[i];
        if (meta_out) meta_out[d] = R.meta[i];
    }
}

int grid_for(uint32_t n, int threads, int cap_blocks)
{
    int b = (int)((n + threads - 1) / threads);
    if (b > cap_blocks) b = cap_blocks;
    return b < 1 ? 1 : b;
}

}  // namespace

int sort_scan_blocks(uint32_t nbins) { return (int)((nbins + kSortScanBlock - 1) / kSortScanBlock); }

cudaError_t launch_sort(const RunDev& R, uint32_t cap, const ParticleSet& dst, uint32_t* hist, uint32_t* off,
                        uint32_t* blk, uint4* aos, cudaStream_t s)
{
    const uint32_t nbins = 2u * R.ncells + 1u;
    const int nb = sort_scan_blocks(nbins);
    k_sort_count<<<grid_for(cap, 256, 8192), 256, 0, s>>>(R, cap, hist);
    k_scan1<<<nb, kSortThreads, 0, s>>>(hist, off, blk, nbins);
    k_scan2<<<1, 1024, 0, s>>>(blk, (uint32_t)nb, off, nbins);
    k_scan3<<<nb, kSortThreads, 0, s>>>(off, blk, nbins);
    if (aos) {
        k_sort_move<true><<<grid_for(cap, 256, 8192), 256, 0, s>>>(R, cap, dst, aos, hist, off);
        k_sort_unpack<<<grid_for(cap, 256, 8192), 256, 0, s>>>(aos, cap, dst);
    } else {
        k_sort_move<false><<<grid_for(cap, 256, 8192), 256, 0, s>>>(R, cap, dst, nullptr, hist, off);
    }
    return cudaGetLastError();
}

cudaError_t launch_export_ordered(const RunDev& R, uint32_t n, uint32_t cap, float* const out[6], uint32_t* meta_out,
                                  double sxy, double sz, cudaStream_t s)
{
    OutPtrs o;
    for (int k = 0; k < 6; ++k) o.p[k] = out ? out[k] : nullptr;
    k_export_ordered<<<grid_for(cap, 256, 8192), 256, 0, s>>>(R, n, cap, o, meta_out, sxy, sz);
    return cudaGetLastError();
}

}  // namespace ecris
