// Internal definitions shared by the CUDA translation units of the ECRIS
// library: the per-run device parameter block, the tally layout and the
// device-side building blocks of the time step (Philox words, field model,
// E-grid gather).  Host-side API code lives in api.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "../../include/ecris.h"

namespace ecris {

constexpr int kQSlots = 64;            // charge-state slots per tally array
#ifndef ECRIS_TILE_VEC
#define ECRIS_TILE_VEC 2
#endif
#ifndef ECRIS_STEP_MIN_BLOCKS
#define ECRIS_STEP_MIN_BLOCKS 5
#endif
constexpr int kThreads = 256;                 // threads per block of the step kernel
constexpr int kVec = ECRIS_TILE_VEC;          // particles per thread per tile
constexpr int kTile = kThreads * kVec;        // particles per tile
constexpr int kTileGroups = kTile / 4;        // float4 groups per tile
constexpr int kStepMinBlocks = ECRIS_STEP_MIN_BLOCKS;   // resident step-kernel blocks per SM asked of ptxas

// Tally words per run (u64): extracted[64], lost[64], kinetic energy of ions
// that left (micro-eV), Coulomb pair collisions.
constexpr int kTallyExtracted = 0;
constexpr int kTallyLost = 64;
constexpr int kTallyKe = 128;
constexpr int kTallyCoulomb = 129;
constexpr int kTallyWords = 132;
// first-passage times: 4 bins per octave of the age in steps (ages < 2^30)
constexpr int kFptdBins = ECRIS_FPTD_BINS;
// [Q][bin] counts, [Q] age sums, [Q] extraction radius sums (nm)
constexpr int kFptdWords = kQSlots * (kFptdBins + 2);
constexpr int kFptdAgeSum = kQSlots * kFptdBins;
constexpr int kFptdRadius = kQSlots * (kFptdBins + 1);

// meta word layout (matches the public header)
constexpr uint32_t kQMask = 0xFFu;
constexpr uint32_t kEvWall = 1u << 8;
constexpr uint32_t kEvExtract = 1u << 9;
constexpr uint32_t kEvIonize = 1u << 10;
constexpr uint32_t kEvCx = 1u << 11;
constexpr uint32_t kEvCoulomb = 1u << 12;
constexpr uint32_t kEvElastic = 1u << 13;
constexpr uint32_t kEvRecomb = 1u << 14;
constexpr uint32_t kStFrozen = 1u << 16;
constexpr uint32_t kStPad = 1u << 17;   // padding slot, never processed

// process switches (match ECRIS_F_*)
constexpr uint32_t kFPush = 1u << 0;
constexpr uint32_t kFIonize = 1u << 1;
constexpr uint32_t kFCx = 1u << 2;
constexpr uint32_t kFEikick = 1u << 3;
constexpr uint32_t kFCoulomb = 1u << 4;
constexpr uint32_t kFRecycle = 1u << 5;
constexpr uint32_t kFIsoheat = 1u << 6;
constexpr uint32_t kFDouble = 1u << 7;
constexpr uint32_t kFElastic = 1u << 8;
constexpr uint32_t kFRecomb = 1u << 9;
constexpr uint32_t kFlagMask = 0x3FFu;
// processes whose code only the variant step kernels carry (with the
// on-axis field table)
constexpr uint32_t kFVariants = kFDouble | kFElastic | kFRecomb;
constexpr uint32_t kFHasE = 1u << 16;   // internal: the run has a nonzero E grid (the push gathers it)

constexpr uint32_t kNoCell = 0xFFFFFFFFu;

// bounded waits: iterations of mbarrier.try_wait before a kernel gives up,
// records ECRIS_ETIMEOUT (4) in the run's error word and stops its work
constexpr uint32_t kWaitLimit = 1u << 20;
constexpr uint32_t kErrTimeout = 4u;

// Nanbu A(s) table: ln A tabulated on a uniform grid in ln s over [1e-3, 6]
constexpr int kNanbuN = 2048;
constexpr double kNanbuSLo = 1e-3;
constexpr double kNanbuSHi = 6.0;

// scan of the per-cell participant counts: cells per scan tile (one block)
constexpr int kScanThreads = 256;
constexpr int kScanPerThread = 8;     // a multiple of 4 (vector loads)
constexpr int kScanBlock = kScanThreads * kScanPerThread;

// Device parameter block of one run: FP32 constants of the kernels (built in
// FP64 on the host) and the run's device arrays.
struct alignas(16) RunDev {
    // geometry
    float R0, R0sq, L, r_ap_sq, eps_wall;
    float inlet_x, inlet_y, inlet_z;
    // fixed-point positions: x = X sxy, y = Y sxy, z = (Z + 2^31) sz for int32
    // X, Y, Z, a uniform grid of 2^32 points across [-R0, R0) and [0, L)
    float sxy, inv_sxy, sz, inv_sz;
    float dt_sxy, dt_sz;         // dt / sxy, dt / sz: displacement per unit velocity
    int32_t inlet_X, inlet_Y, inlet_Z;   // gas inlet in fixed point
    // FP64 geometry for the (rare) wall and aperture crossings
    double R0_d, L_d, r_ap_d, eps_wall_d, sxy_d, sz_d;
    // synthetic mirror B0(z): raised-cosine halves around z_m
    float B_min, aL, aR;         // half amplitudes (B_inj-B_min)/2, (B_ext-B_min)/2
    float zm, inv_zm, inv_zr;    // z_m, 1/z_m, 1/(L-z_m)
    float aLk, aLk2, aRk, aRk2;  // a k and a k^2 of each half (k = pi/z_m, pi/(L-z_m))
    float hex_c;                 // B_hex / R0^2
    // on-axis table instead of the mirror: per segment k of length h the cubic
    // B0 = a + t (b + t (c + t d)), t = z/h - k (nullptr: the mirror)
    const float4 *btab;
    int32_t nseg;
    float inv_h;
    float B_ecr;
    // mesh
    int32_t nx, ny, nz;
    float inv_dx, inv_dy, inv_dz;
    // species and push
    int32_t qmax;
    float qm_unit;               // e / (M amu)
    float dt, half_dt;
    // collisions
    uint32_t flags;
    float sig0;                  // sqrt(kT0/M): thermal speed of re-emitted atoms
    float n0s1;                  // n0 * sigma_1 (1/m)
    float vth2;                  // 8 kT0 / (pi M)
    float dv_cx;                 // kick of a Q>=3 charge exchange: sqrt(2 (E_cx/2) / M)
    float n0sel;                 // n0 * sigma_el1 (1/m): elastic ion-atom scattering
    float sig_refl;              // thermal speed of ions re-emitted after neutralisation at a wall
    float ei_coef[2];            // D^2 = ei_coef[zone] * n_e * Q^p (zone 0 cold, 1 warm)
    int32_t ei_pow;
    float ke_scale;              // (M/2) / e * 1e6: micro-eV per (m/s)^2
    uint32_t atom_gate;          // an atom whose ionisation word is >= atom_gate cannot ionise in
                                 // any cell (0xFFFFFFFF: no such bound); 0: read the gate the device
                                 // keeps after the rate table (set by a device update of n_e)
    float lnl_ii_coef;           // Nanbu s prefactor lnL/(4 pi) (e^2/(eps0 mu))^2 w / V_cell
    uint32_t seed_lo, seed_hi;
    // arrays
    int32_t *x, *y, *z;          // fixed-point positions (see sxy, sz)
    float *vx, *vy, *vz;
    uint32_t *meta;
    uint32_t *id;                // stable particle id (Philox counter word, output order)
    const float4 *cell;          // {n_e (m^-3), zone (0/1), delta_x, delta_y}
    const float4 *E;             // {E_x, E_y, E_z, 0} per cell centre
    const float *kdt;            // [zone * 64 + Q]: k dt with k = k1 (single ionisation) + k2 (double)
                                 // + k3 (triple) + kr (recombination) as switched on; then
                                 // [2 * 64 + ...] the share k1 / k, [4 * 64 + ...] the share
                                 // (k1 + k2) / k and [6 * 64 + ...] (k1 + k2 + k3) / k; then at
                                 // kGateWord the atom gate (uint32 bits): an atom whose ionisation
                                 // word is >= the gate cannot ionise in any cell (0xFFFFFFFF: no
                                 // such bound), and the largest n_e of the cold and warm cells
    unsigned long long *dep;     // packed deposit accumulator: count << 32 | charge
    unsigned long long *tally;   // kTallyWords
    uint4 *plist;                // Coulomb participants of each tile: (slot, cell, id, 0), `tile` slots a tile
    float4 *pvel;                // their (vx, vy, vz, Q as bits), same slots
    uint32_t *tcount;            // participants per tile
    uint32_t *ccount;            // Coulomb participants per cell (counted up by the step kernel,
                                 // counted back to zero by the scatter)
    uint32_t *coff;              // exclusive scan of ccount, Nc + 1 entries
    unsigned long long *cstat;   // scan tile status words (decoupled look-back), one per scan tile
    unsigned long long *cctr;    // scan tile tickets handed out so far
    uint32_t *cstart;            // first participant of each collision range (a range holds whole cells)
    uint32_t *crange;            // [0] participants per range this step, [1] largest cell count seen by
                                 // this step's scan (sets the next step's range size)
    unsigned long long *ckeys;   // (pairing hash << 32 | pid) per participant, grouped by cell
    float4 *crec;                // (vx, vy, vz, cell << 6 | Q as bits) per participant, grouped by cell
    uint32_t *cslot;             // array slot of each participant, grouped by cell
    uint32_t *sslot;             // scratch: pairing order of a range of cells too large for shared memory
    const float *nanbu;          // ln A at ln s = nanbu_lnlo + i / nanbu_inv_dln, i < kNanbuN
    float nanbu_lnlo, nanbu_inv_dln;
    uint32_t *step;              // device step counter of the run
    uint32_t *leave;             // slots of the particles that left the chamber this step
    uint32_t *nleave;            // their number (zero between steps)
    uint32_t *err;               // device error word: 0, or ECRIS_ETIMEOUT after a bounded wait ran out
    uint32_t *birth;             // by particle id: step of the last ionisation from Q = 0 (~0: unknown)
    unsigned long long *fptd;    // [Q][kFptdBins] extraction counts by age bin, [Q] summed ages (steps),
                                 // [Q] summed extraction radii (nm)
    uint32_t n;                  // particles
    uint32_t n4;                 // float4 groups = ceil(n/4)
    uint32_t ncells;
    uint32_t tile;               // particles per tile of the step kernel's launch shape
};

// ----------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11), counter (c0, 0, c2, 0), key (k0, k1).
// ----------------------------------------------------------------------------
struct Words { uint32_t w0, w1, w2, w3; };

__device__ __forceinline__ Words philox(uint32_t c0, uint32_t c2, uint32_t k0, uint32_t k1)
{
    uint32_t c1 = 0u, c3 = 0u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32x32 -> 64-bit product gives both halves
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return Words{c0, c1, c2, c3};
}

// words of particle pid at step s, stream st: counter (pid, 0, 4 s + st, 0)
__device__ __forceinline__ Words rng_words(const RunDev& R, uint32_t pid, uint32_t step, uint32_t st)
{
    return philox(pid, step * 4u + st, R.seed_lo, R.seed_hi);
}

// Programmatic dependent launch: a kernel launched with launch_pdl may be
// scheduled while the kernel before it in the stream finishes (that kernel's
// blocks signal with pdl_trigger, or by exiting); it calls pdl_wait before it
// touches memory, which waits until the kernel before it has completed and
// its writes are visible.  This hides the launch latency between the
// dependent kernels of a step.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// square root through the approximate hardware instruction (relative error
// of a few units in the last place): for quantities that only set a
// probability, the size of a random kick or a scattering geometry, where that
// error is far below the parity tolerance; the push itself uses no square root
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// (cos, sin)(2 pi u) for u in (0, 1] through the fast intrinsic, its argument
// kept inside [-pi, pi] where the absolute error is below 2^-21:
// (cos, sin)(2 pi u) = -(cos, sin)(pi (2u - 1))
__device__ __forceinline__ void sincos_2pi(float u, float* s, float* c)
{
    float sp, cp;
    __sincosf(3.14159265358979f * (2.0f * u - 1.0f), &sp, &cp);
    *s = -sp;
    *c = -cp;
}

// uniform in (0, 1]: (top 24 bits + 1) * 2^-24, exact in FP32
__device__ __forceinline__ float unit01(uint32_t w)
{
    return (float)((w >> 8) + 1u) * (1.0f / 16777216.0f);
}

// event test: fires when the word is below floor(p * 2^32)
__device__ __forceinline__ bool fires(uint32_t w, float p)
{
    const float t = p * 4294967296.0f;
    if (t >= 4294967296.0f) return true;
    return w < __float2uint_rz(t);
}

// ----------------------------------------------------------------------------
// Static magnetic field: synthetic mirror, paraxial off axis, plus the
// hexapole B_H (2xy, x^2 - y^2) / R0^2 (the printed sin/cos(2 theta) R^2 form).
// ----------------------------------------------------------------------------
__device__ __forceinline__ void bfield(const RunDev& R, float x, float y, float z,
                                       float& Bx, float& By, float& Bz)
{
    float b0, b1, b2, s, c;
    if (z <= R.zm) {
        __sincosf(3.14159265358979f * (z * R.inv_zm), &s, &c);   // argument in [0, pi]
        b0 = fmaf(R.aL, 1.0f + c, R.B_min);
        b1 = -R.aLk * s;
        b2 = -R.aLk2 * c;
    } else {
        __sincosf(3.14159265358979f * ((z - R.zm) * R.inv_zr), &s, &c);
        b0 = fmaf(R.aR, 1.0f - c, R.B_min);
        b1 = R.aRk * s;
        b2 = R.aRk2 * c;
    }
    // (FMAs written out: the step kernel is compiled without contraction)
    const float hx = -0.5f * b1, hz = -0.25f * b2;
    const float r2 = fmaf(x, x, y * y);
    Bx = fmaf(hx, x, R.hex_c * (2.0f * x * y));
    By = fmaf(hx, y, R.hex_c * fmaf(x, x, -y * y));
    Bz = fmaf(hz, r2, b0);
}

// the same from the on-axis table: the segment's cubic in t and its
// derivatives in z
__device__ __forceinline__ void bfield_table(const RunDev& R, float x, float y, float z,
                                             float& Bx, float& By, float& Bz)
{
    const float u = z * R.inv_h;
    int k = (int)u;
    k = k < 0 ? 0 : (k > R.nseg - 1 ? R.nseg - 1 : k);
    const float t = u - (float)k;
    const float4 cf = __ldg(R.btab + k);
    const float b0 = cf.x + t * (cf.y + t * (cf.z + t * cf.w));
    const float b1 = (cf.y + t * (2.0f * cf.z + 3.0f * t * cf.w)) * R.inv_h;
    const float b2 = (2.0f * cf.z + 6.0f * t * cf.w) * (R.inv_h * R.inv_h);
    const float r2 = x * x + y * y;
    Bx = -0.5f * x * b1 + R.hex_c * (2.0f * x * y);
    By = -0.5f * y * b1 + R.hex_c * (x * x - y * y);
    Bz = b0 - 0.25f * r2 * b2;
}

// one axis of the trilinear gather between cell centres, clamped at the faces
__device__ __forceinline__ void tri_axis(float g, int n, int& i0, float& f)
{
    const float gc = g - 0.5f;
    const float fl = floorf(gc);
    int i = (int)fl;
    if (i < 0) { i0 = 0; f = 0.0f; }
    else if (i > n - 2) { i0 = n - 2; f = 1.0f; }
    else { i0 = i; f = gc - fl; }
}

__device__ __forceinline__ void efield(const RunDev& R, float x, float y, float z,
                                       float& Ex, float& Ey, float& Ez)
{
    int ix, iy, iz;
    float fx, fy, fz;
    tri_axis((x + R.R0) * R.inv_dx, R.nx, ix, fx);
    tri_axis((y + R.R0) * R.inv_dy, R.ny, iy, fy);
    tri_axis(z * R.inv_dz, R.nz, iz, fz);
    const int sx = 1, sy = R.nx, sz = R.nx * R.ny;
    const float4* e = R.E + ((iz * R.ny + iy) * R.nx + ix);
    const float4 a000 = __ldg(e), a100 = __ldg(e + sx), a010 = __ldg(e + sy), a110 = __ldg(e + sy + sx);
    const float4 a001 = __ldg(e + sz), a101 = __ldg(e + sz + sx), a011 = __ldg(e + sz + sy),
                 a111 = __ldg(e + sz + sy + sx);
    const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
    const float w000 = gx * gy * gz, w100 = fx * gy * gz, w010 = gx * fy * gz, w110 = fx * fy * gz;
    const float w001 = gx * gy * fz, w101 = fx * gy * fz, w011 = gx * fy * fz, w111 = fx * fy * fz;
    Ex = w000 * a000.x + w100 * a100.x + w010 * a010.x + w110 * a110.x +
         w001 * a001.x + w101 * a101.x + w011 * a011.x + w111 * a111.x;
    Ey = w000 * a000.y + w100 * a100.y + w010 * a010.y + w110 * a110.y +
         w001 * a001.y + w101 * a101.y + w011 * a011.y + w111 * a111.y;
    Ez = w000 * a000.z + w100 * a100.z + w010 * a010.z + w110 * a110.z +
         w001 * a001.z + w101 * a101.z + w011 * a011.z + w111 * a111.z;
}

// fixed point <-> metres
__device__ __forceinline__ float fx_xy(const RunDev& R, int32_t X) { return (float)X * R.sxy; }
__device__ __forceinline__ float fx_z(const RunDev& R, int32_t Z) { return ((float)Z + 2147483648.0f) * R.sz; }
__device__ __forceinline__ int32_t to_fx_xy(const RunDev& R, float x) { return __float2int_rn(x * R.inv_sxy); }
__device__ __forceinline__ int32_t to_fx_z(const RunDev& R, float z)
{
    return (int32_t)(__float2uint_rn(z * R.inv_sz) ^ 0x80000000u);
}

// nearest-grid-point cell of a fixed-point position: with U = X + 2^31 the
// cell is floor(U n / 2^32), the high word of a 32x32-bit product (exact)
__device__ __forceinline__ uint32_t ngp_cell(const RunDev& R, int32_t X, int32_t Y, int32_t Z)
{
    const uint32_t ix = __umulhi((uint32_t)X ^ 0x80000000u, (uint32_t)R.nx);
    const uint32_t iy = __umulhi((uint32_t)Y ^ 0x80000000u, (uint32_t)R.ny);
    const uint32_t iz = __umulhi((uint32_t)Z ^ 0x80000000u, (uint32_t)R.nz);
    return (iz * (uint32_t)R.ny + iy) * (uint32_t)R.nx + ix;
}

// moment probes and screens (probe.cu)
constexpr int kMaxScreens = ECRIS_MAX_SCREENS;
struct ProbeDev {
    const int32_t* slot;          // per cell: its probe slot, or -1 (nullptr: no probed cells)
    double* mom;                  // [slot][qs][7]: count, sums of v and of v^2 per component
    unsigned long long* screen;   // [screen][qs][pixels^2] hit counts
    uint32_t ulo[kMaxScreens];    // slab of each screen in U = Z + 2^31: ulo <= U <= uhi
    uint32_t uhi[kMaxScreens];
    int32_t nscreens;
    int32_t pix_log2;             // pixels = 2^pix_log2
    int32_t qs;                   // qmax + 1
};

// ----------------------------------------------------------------------------
// Launch wrappers (defined in step_kernel.cu / coulomb.cu)
// ----------------------------------------------------------------------------
// one pass of the fused step kernel over the run's ntiles tiles of kTile
// particles; the particles that left the chamber are listed in R.leave
cudaError_t launch_step(const RunDev& R, uint32_t ntiles, int grid, cudaStream_t s);
// the leaver pass after it: crossing, tallies, re-emission and deposit of the
// listed particles; the list is cleared; bump_step: advance the step counter
// (ticket: a zeroed device word, left zero)
constexpr int kLeaveBlocks = 64;
cudaError_t launch_leave(const RunDev& R, unsigned int* ticket, int bump_step, cudaStream_t s);
// the same for every run of a batch (step counters untouched)
cudaError_t launch_leave_batch(const RunDev* runs, uint32_t nruns, unsigned int* ticket, cudaStream_t s);
cudaError_t launch_fold(const RunDev& R, uint32_t ncells, unsigned long long* count,
                        unsigned long long* charge, cudaStream_t s);
// words of the rate table after its 8 kQSlots rates and shares: the atom gate and the
// FP32 bits of the largest n_e of the cold and the warm cells
constexpr int kGateWord = 8 * kQSlots;
constexpr int kKdtWords = kGateWord + 4;
// the atom gate from the rate table's k_0 dt and the stored largest n_e of
// each zone (ne_update.cu)
cudaError_t launch_atom_gate(float* kdt, cudaStream_t s);
// self-consistent n_e: every cell's n_e from the charge deposited since the
// mark over steps_vol = steps V_cell, the mark moved on, the records {n_e,
// zone, delta} rebuilt (rl_coef = 2.38e-6 sqrt(T_e)/(B dX) per cell) and the
// atom gate recomputed; ne (Nc doubles) is scratch
cudaError_t launch_ne_update(const unsigned long long* charge, unsigned long long* mark, double* ne,
                             const double* rl_coef, float4* cell, float* kdt, int nx, int ny, uint32_t ncells,
                             double weight, double steps_vol, bool isoheat, int sm_count, cudaStream_t s);
// validity limits and padding point for ecris_load_ions
struct LoadCheck {
    float R0sq, L;
    uint32_t qmax;
    float inlet_x, inlet_y, inlet_z;
    float inv_sxy_hi, inv_sxy_lo;   // metres -> fixed point, as an unevaluated FP32 sum
    float inv_sz_hi, inv_sz_lo;
};
// check particles [0, n), convert their positions (metres, float) in place to
// fixed point, build their meta words from q8 and ids, fill pads [n, cap);
// bad[0] counts invalid particles, bad[1] holds the lowest invalid index
cudaError_t launch_load_init(const LoadCheck& lc, float* const soa[6], const uint8_t* q8, uint32_t* meta,
                             uint32_t* id, uint32_t n, uint32_t cap, unsigned int* bad, cudaStream_t s);

// One set of particle arrays (the sort moves particles between two sets).
struct ParticleSet {
    int32_t *x, *y, *z;
    float *vx, *vy, *vz;
    uint32_t *meta, *id;
};
// Counting sort of the run's particles (in R) by (ion/atom, cell) into `dst`:
// live ions first, then live atoms, each by cell; frozen and padding slots
// last.  hist (2 Nc + 1 words) must be zero and is left zero; off (2 Nc + 2)
// and blk (scan block totals) are scratch.  aos (2 cap uint4 of scratch, or
// NULL): move through 32-byte records, for input in arbitrary order (the
// first sort after a load); NULL writes the destination arrays directly.
cudaError_t launch_sort(const RunDev& R, uint32_t cap, const ParticleSet& dst, uint32_t* hist, uint32_t* off,
                        uint32_t* blk, uint4* aos, cudaStream_t s);
int sort_scan_blocks(uint32_t nbins);
// state in load order: out[id[slot]] = state[slot] for id < n (positions to
// metres), into device arrays
cudaError_t launch_export_ordered(const RunDev& R, uint32_t n, uint32_t cap, float* const out[6], uint32_t* meta_out,
                                  double sxy, double sz, cudaStream_t s);
cudaError_t launch_census(const RunDev& R, uint32_t n4, unsigned long long* census, cudaStream_t s);
// add the current particles to the probes' sums (probe.cu)
cudaError_t launch_probe(const RunDev& R, const ProbeDev& P, uint32_t n4, int sm_count, cudaStream_t s);

// resident blocks per SM of the step kernel
int step_blocks_per_sm();
// Launch shapes of the batched step kernel: threads per block x particles per
// thread and tile, shape k = (kShapeThreads[k], kShapeVec[k]); tile sizes
// from 128 to 2048 particles
constexpr int kStepShapes = 12;
constexpr int kDefaultShape = 11;   // 256 x 2 with three stages
constexpr int kShapeThreads[kStepShapes] = {128, 128, 128, 256, 256, 256, 512, 512, 512, 128, 256, 256};
constexpr int kShapeVec[kStepShapes] = {1, 2, 4, 1, 2, 4, 1, 2, 4, 2, 1, 2};
constexpr int kShapeStages[kStepShapes] = {2, 2, 2, 2, 2, 2, 2, 2, 2, 3, 3, 3};
constexpr int kMinTile = 128, kMaxTile = 2048;
inline uint32_t shape_tile(int k) { return (uint32_t)(kShapeThreads[k] * kShapeVec[k]); }
int step_batch_blocks_per_sm(int shape);
// batch form: one persistent step-kernel launch over the work items (run,
// tile) of many runs whose parameter blocks are in device memory (it leaves
// the step counters alone); the batch leaver pass then advances the counters
// of the runs without Coulomb collisions (the collision kernels of the
// others, launched after it, advance theirs); entries with step == NULL are
// skipped
// variants: launch the kernel with the opt-in processes' code (some run has
// one of kFVariants)
cudaError_t launch_step_batch(const RunDev* runs, const uint2* items, uint32_t nitems, int grid, bool variants,
                              int shape, cudaStream_t s);
// message returned by ecris_last_error(NULL) on the calling thread
void ecris_internal_set_thread_error(const char* msg);
// host: ln A(s) of Nanbu's scattering law on kNanbuN points uniform in ln s
// over [kNanbuSLo, kNanbuSHi], built in FP64 once per process (api.cu)
const float* nanbu_table();
// host: the prefactor of Nanbu's s = coef Qa^2 Qb^2 m g^-3 dt for m ions of
// one cell: lnL/(4 pi) (e^2/(eps0 mu))^2 w / V_cell, mu = M/2 (api.cu)
float coulomb_s_coef(double lnL_ii, double mass_amu, double weight, double cell_volume_m3);

// Hooks of the served form (defined in api.cu, used by server.cu).  A tally
// snapshot is a run's tally words and device error word, copied in stream
// order into pinned host memory at a step boundary; the served loop reads it
// a tick later, while the batch keeps stepping.
struct TallySnapshot {
    unsigned long long tally[kTallyWords];
    uint32_t err, pad;
};
// enqueue the copies of run `run`'s tallies into *dst (pinned) on the batch stream
ecris_status batch_snapshot(ecris_batch* b, int32_t run, TallySnapshot* dst);
cudaStream_t batch_stream(const ecris_batch* b);
// the batch autotuner (ecris_batch_autotune); without `cadence` it keeps the
// sort cadence and times launch shapes and resident blocks only
ecris_status batch_autotune(ecris_batch* b, uint32_t trial_steps, bool cadence, ecris_tuning* chosen);
// fill out (extracted, lost, currents, power, wall energy, collisions) from a
// snapshot taken after `steps` steps of the run (time steps * dt)
void batch_snapshot_diag(const ecris_batch* b, int32_t run, const TallySnapshot& snap, uint64_t steps,
                         ecris_diag_out* out);

// Coulomb collisions of one run for the current step, after the step
// kernel: scan of the cell counts, scatter of the pairing keys, and the
// per-cell sort / pair / collide kernel, whose last block advances the step
// counter and clears the leaver list.  leave_blocks extra blocks of the scan
// kernel (the same count at every launch of a run: kLeaveBlocks for one run,
// 0 in a batch) run the step's leaver pass if do_leave, in place of
// launch_leave; else the leavers were finished before, by launch_leave or
// the batch's pass.
constexpr int kCoulombKernels = 3;   // kernels per launch_coulomb
// participants per range of cells of the collision kernel: the first step
// after a load takes kCellIons; each later step takes kCellCap minus the
// largest cell count of the step before, within [kCellIonsMin, kCellIonsMax],
// so that a range (its cells whole) still fits in shared memory while ranges
// stay as large as it allows (fewer ranges, fewer per-range waits)
constexpr int kCellIons = 512;
constexpr int kCellIonsMin = 256, kCellIonsMax = 896;
constexpr int kCellCap = 1024;       // participants of a range held in shared memory
cudaError_t launch_coulomb(const RunDev& R, uint32_t ncells, uint32_t ntiles, unsigned int* ticket, int grid,
                           uint32_t leave_blocks, int do_leave, cudaStream_t s);
// the cell-count scan of the collisions, with leave_blocks extra blocks for
// the leaver pass (step_kernel.cu)
cudaError_t launch_scan(const RunDev& R, uint32_t ncells, uint32_t nscan, uint32_t leave_blocks, int do_leave,
                        cudaStream_t s);
int coulomb_scan_blocks(uint32_t ncells);
int collide_blocks_per_sm();

}  // namespace ecris
