// ecris_coulomb_collide_noalloc: one ion-ion Coulomb collision step (the same
// Takizawa-Abe pairing and Nanbu scattering kernels ecris_step runs) for a
// caller that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they need a collision
// step: code inside a region where the CUDA caching or stream-ordered
// allocators are off limits, embedded or real-time hosts that reserve all
// device memory up front and forbid allocation afterwards, and plug-ins
// running inside a larger simulation whose memory manager owns the device.
// cudaMalloc can also synchronise the device, which such callers must avoid.
// This entry point therefore keeps all its working memory (per-cell counts and
// offsets, participant records and keys, the Nanbu table, counters) in one
// file-scope device array of fixed size, and allocates nothing.
//
// Limits: at most kNaMaxIons particles and kNaMaxCells cells per call; larger
// sizes are rejected with ECRIS_EINVAL.  The array (kNaScratchBytes, about
// 4.5 MB) is held by every GPU that loads the library until the process exits.
// Every call shares it and finds the last call's contents there; what must
// start at zero is cleared at the start of each call.  Calls whose GPU work
// overlaps (different streams, or several host threads) race on the array
// and must be serialised by the caller.  The first call on each device sets up
// that device (symbol address, Nanbu table upload, a synchronous copy); make
// that first call before any stream capture begins.  That set-up is kept for
// the life of the process: a device reset (cudaDeviceReset) is not supported,
// and the entry point must not be called on a device after one.
// A bounded wait inside the cell-count scan that runs out (possible only when
// calls overlap) sets an error word in the array instead of faulting; a call
// given collisions_out synchronises, reads that word and returns
// ECRIS_ETIMEOUT.  A call without collisions_out returns at once and does not
// report it.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ecris.h"
#include "ecris_internal.cuh"

using namespace ecris;

namespace {

constexpr uint32_t kNaMaxIons = 65536;
constexpr uint32_t kNaMaxCells = 65536;
constexpr uint32_t kNaTiles = kNaMaxIons / kTile;
constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// byte offsets of the sub-buffers inside the scratch array
constexpr size_t kOffPlist = 0;
constexpr size_t kOffPvel = kOffPlist + align256(sizeof(uint4) * kNaMaxIons);
constexpr size_t kOffTcount = kOffPvel + align256(sizeof(float4) * kNaMaxIons);
constexpr size_t kOffCcount = kOffTcount + align256(sizeof(uint32_t) * kNaTiles);
constexpr size_t kOffCoff = kOffCcount + align256(sizeof(uint32_t) * kNaMaxCells);
constexpr uint32_t kNaScanTiles = kNaMaxCells / kScanBlock + 1;
constexpr size_t kOffCstat = kOffCoff + align256(sizeof(uint32_t) * (kNaMaxCells + 1));
constexpr size_t kOffCkeys = kOffCstat + align256(sizeof(unsigned long long) * (kNaScanTiles + 1));
constexpr size_t kOffCrec = kOffCkeys + align256(sizeof(unsigned long long) * kNaMaxIons);
constexpr size_t kOffCslot = kOffCrec + align256(sizeof(float4) * kNaMaxIons);
constexpr size_t kOffSslot = kOffCslot + align256(sizeof(uint32_t) * kNaMaxIons);
constexpr size_t kOffCstart = kOffSslot + align256(sizeof(uint32_t) * kNaMaxIons);
constexpr size_t kOffNanbu = kOffCstart + align256(sizeof(uint32_t) * (kNaMaxIons / kCellIonsMin + 2));
constexpr size_t kOffWords = kOffNanbu + align256(sizeof(float) * kNanbuN);
// words: step, ticket, error word, -, collision range size and largest cell count; then the tally block
constexpr size_t kOffTally = kOffWords + 256;
constexpr size_t kNaScratchBytes = kOffTally + align256(sizeof(unsigned long long) * kTallyWords);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

struct DeviceSetup {
    bool ready = false;
    unsigned char* base = nullptr;   // device address of g_noalloc_scratch
    int grid = 0;
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[64];

// clear the per-call counters and store the step index
__global__ void k_na_init(unsigned char* base, uint32_t ncells, uint32_t tiles, uint32_t step)
{
    uint32_t* ccount = reinterpret_cast<uint32_t*>(base + kOffCcount);
    uint32_t* tcount = reinterpret_cast<uint32_t*>(base + kOffTcount);
    uint32_t* words = reinterpret_cast<uint32_t*>(base + kOffWords);
    unsigned long long* tally = reinterpret_cast<unsigned long long*>(base + kOffTally);
    unsigned long long* cstat = reinterpret_cast<unsigned long long*>(base + kOffCstat);
    const uint32_t stride = gridDim.x * blockDim.x;
    // scan status words and their ticket counter (the scan's tile count
    // changes with ncells from call to call)
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= kNaScanTiles; i += stride) cstat[i] = 0ull;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ncells; i += stride) ccount[i] = 0u;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < tiles; i += stride) tcount[i] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        words[0] = step;
        words[1] = 0u;   // the collision kernel's ticket
        words[2] = 0u;   // error word: the scan sets ECRIS_ETIMEOUT if a bounded wait runs out
        words[4] = (uint32_t)kCellIons;   // collision range size of this call
        words[5] = 0u;
    }
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (uint32_t)kTallyWords; i += stride) tally[i] = 0ull;
}

// publish the participants (cell < ncells, Q >= 1) in their tile's list and
// count them per cell, as the fused step kernel does for ecris_step
__global__ void k_na_pack(unsigned char* base, uint32_t n, const uint32_t* __restrict__ cell,
                          const uint8_t* __restrict__ q, const float* __restrict__ vx,
                          const float* __restrict__ vy, const float* __restrict__ vz, uint32_t ncells)
{
    uint4* plist = reinterpret_cast<uint4*>(base + kOffPlist);
    float4* pvel = reinterpret_cast<float4*>(base + kOffPvel);
    uint32_t* tcount = reinterpret_cast<uint32_t*>(base + kOffTcount);
    uint32_t* ccount = reinterpret_cast<uint32_t*>(base + kOffCcount);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t c = cell[i];
        const uint32_t Q = q[i];
        if (c >= ncells || Q == 0u || Q > 63u) continue;
        const uint32_t t = i / kTile;
        const uint32_t slot = t * kTile + atomicAdd(tcount + t, 1u);
        plist[slot] = make_uint4(i, c, i, 0u);   // slot and id are both the array index
        pvel[slot] = make_float4(vx[i], vy[i], vz[i], __uint_as_float(Q));
        atomicAdd(ccount + c, 1u);
    }
}

ecris_status na_fail(const std::string& msg)
{
    ecris_internal_set_thread_error(msg.c_str());
    return ECRIS_EINVAL;
}

ecris_status na_cuda(cudaError_t e, const char* what)
{
    ecris_internal_set_thread_error((std::string("coulomb_collide_noalloc: ") + what + ": " +
                                     cudaGetErrorString(e)).c_str());
    return ECRIS_ECUDA;
}

}  // namespace

extern "C" ecris_status ecris_coulomb_collide_noalloc(size_t n, const uint32_t* cell, const uint8_t* q, float* vx,
                                                      float* vy, float* vz, uint32_t* events, uint32_t ncells,
                                                      double mass_amu, double weight, double cell_volume_m3,
                                                      double lnL_ii, double dt, uint64_t seed, uint32_t step,
                                                      void* cuda_stream, int64_t* collisions_out)
{
    if (n > kNaMaxIons || ncells > kNaMaxCells || ncells == 0)
        return na_fail("coulomb_collide_noalloc: need n <= " + std::to_string(kNaMaxIons) + " and 1 <= ncells <= " +
                       std::to_string(kNaMaxCells) + " (fixed scratch size)");
    if (n > 0 && (!cell || !q || !vx || !vy || !vz || !events))
        return na_fail("coulomb_collide_noalloc: NULL array");
    if (!(mass_amu > 0.0) || !(weight > 0.0) || !(cell_volume_m3 > 0.0) || !(lnL_ii >= 0.0) || !(dt > 0.0) ||
        !std::isfinite(mass_amu) || !std::isfinite(weight) || !std::isfinite(cell_volume_m3) ||
        !std::isfinite(lnL_ii) || !std::isfinite(dt))
        return na_fail("coulomb_collide_noalloc: mass, weight, cell volume and dt must be finite and > 0");
    if ((uint64_t)step * 4u + 3u > 0xFFFFFFFFull) return na_fail("coulomb_collide_noalloc: step must be < 2^30");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_cuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return na_fail("coulomb_collide_noalloc: device index above 63");
    DeviceSetup setup;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        DeviceSetup& d = g_setup[dev];
        if (!d.ready) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return na_cuda(e, "cudaGetSymbolAddress");
            // the same FP64-built table ecris_init_fields uploads for ecris_step
            e = cudaMemcpy(static_cast<unsigned char*>(p) + kOffNanbu, nanbu_table(), kNanbuN * sizeof(float),
                           cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return na_cuda(e, "Nanbu table upload");
            int sms = 0;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return na_cuda(e, "cudaDeviceGetAttribute");
            d.base = static_cast<unsigned char*>(p);
            d.grid = sms * collide_blocks_per_sm();
            d.ready = true;
        }
        setup = d;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned char* base = setup.base;
    const uint32_t tiles = (uint32_t)((n + kTile - 1) / kTile);

    // the parameter block the collision kernels read, pointing into the scratch
    RunDev R;
    std::memset(&R, 0, sizeof R);
    R.lnl_ii_coef = coulomb_s_coef(lnL_ii, mass_amu, weight, cell_volume_m3);
    R.dt = (float)dt;
    R.seed_lo = (uint32_t)seed;
    R.seed_hi = (uint32_t)(seed >> 32);
    R.vx = vx;
    R.vy = vy;
    R.vz = vz;
    R.meta = events;
    R.plist = reinterpret_cast<uint4*>(base + kOffPlist);
    R.pvel = reinterpret_cast<float4*>(base + kOffPvel);
    R.tcount = reinterpret_cast<uint32_t*>(base + kOffTcount);
    R.ccount = reinterpret_cast<uint32_t*>(base + kOffCcount);
    R.coff = reinterpret_cast<uint32_t*>(base + kOffCoff);
    R.cstat = reinterpret_cast<unsigned long long*>(base + kOffCstat);
    R.cctr = R.cstat + kNaScanTiles;
    R.cstart = reinterpret_cast<uint32_t*>(base + kOffCstart);
    R.crange = reinterpret_cast<uint32_t*>(base + kOffWords) + 4;
    R.ckeys = reinterpret_cast<unsigned long long*>(base + kOffCkeys);
    R.crec = reinterpret_cast<float4*>(base + kOffCrec);
    R.cslot = reinterpret_cast<uint32_t*>(base + kOffCslot);
    R.sslot = reinterpret_cast<uint32_t*>(base + kOffSslot);
    R.tile = (uint32_t)kTile;   // the participant lists of k_na_pack, kTile slots a tile
    R.nanbu = reinterpret_cast<const float*>(base + kOffNanbu);
    R.nanbu_lnlo = (float)std::log(kNanbuSLo);
    R.nanbu_inv_dln = (float)((kNanbuN - 1) / std::log(kNanbuSHi / kNanbuSLo));
    R.step = reinterpret_cast<uint32_t*>(base + kOffWords);
    R.err = reinterpret_cast<uint32_t*>(base + kOffWords) + 2;
    R.tally = reinterpret_cast<unsigned long long*>(base + kOffTally);
    unsigned int* ticket = reinterpret_cast<unsigned int*>(base + kOffWords) + 1;

    const uint32_t span = ncells > tiles ? ncells : tiles;
    k_na_init<<<(span + 255) / 256 > 0 ? (span + 255) / 256 : 1, 256, 0, s>>>(base, ncells, tiles, step);
    if (n > 0)
        k_na_pack<<<(uint32_t)((n + 255) / 256), 256, 0, s>>>(base, (uint32_t)n, cell, q, vx, vy, vz, ncells);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_cuda(e, "launch");
    e = launch_coulomb(R, ncells, tiles, ticket, setup.grid, 0u, 0, s);
    if (e != cudaSuccess) return na_cuda(e, "launch_coulomb");
    if (collisions_out) {
        // the call synchronises: read the collision count and the error word
        unsigned long long c = 0;
        uint32_t err = 0;
        e = cudaMemcpyAsync(&c, R.tally + kTallyCoulomb, sizeof c, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&err, R.err, sizeof err, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return na_cuda(e, "collision count");
        if (err != 0u) {
            ecris_internal_set_thread_error(
                "coulomb_collide_noalloc: a bounded wait of the cell-count scan ran out (a call overlapping "
                "this one on the GPU?); the velocities of this call are not valid");
            return ECRIS_ETIMEOUT;
        }
        *collisions_out = (int64_t)c;
    }
    return ECRIS_OK;
}
