// Host side of the C ABI declared in include/ecris.h: validation, FP64 run
// setup (rates, ECR zone, electron density and delta per cell), device memory
// (stream-ordered, owned by the context), kernel launches and diagnostics.
//
// Model: Mironov et al., arXiv:1507.03392, Sec. II.  The FP64 set-up here is
// written independently of any test oracle: the rate of Q -> Q+1 uses the
// closed form of the Maxwellian-averaged single-term Lotz cross section,
//   k = sqrt(8 e / (pi m_e)) a q E1(P/T) / ((P/T) T^1.5),  a = 4.5e-14 cm^2 eV^2,
// with E1 from its power series (x <= 1) and continued fraction (x > 1).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ecris.h"
#include "ecris_internal.cuh"

using namespace ecris;

namespace {

constexpr double kE = 1.602176634e-19;       // C
constexpr double kAmu = 1.66053906660e-27;   // kg
constexpr double kMe = 9.1093837015e-31;     // kg
constexpr double kEps0 = 8.8541878128e-12;   // F/m
constexpr double kPi = 3.14159265358979323846;
constexpr double kLotzA = 4.5e-18;           // m^2 eV^2
constexpr uint32_t kMaxSteps = 1u << 30;     // RNG counter word 2 holds 4*step + stream

thread_local std::string g_create_error;

// Exponential integral E1(x), x > 0 (Abramowitz & Stegun 5.1.11 and 5.1.22).
double expint_e1(double x)
{
    if (x <= 1.0) {
        const double euler = 0.57721566490153286061;
        double sum = 0.0, term = 1.0;
        for (int k = 1; k < 200; ++k) {
            term *= -x / k;                 // (-x)^k / k!
            const double add = term / k;
            sum += add;
            if (std::fabs(add) < 1e-18 * std::fabs(sum)) break;
        }
        return -euler - std::log(x) - sum;
    }
    // modified Lentz evaluation of E1(x) = e^-x / (x + 1 - 1^2/(x + 3 - 2^2/(x + 5 - ...)))
    const double tiny = 1e-300;
    double b = x + 1.0, c = 1.0 / tiny, d = 1.0 / b, h = d;
    for (int i = 1; i < 1000; ++i) {
        const double a = -(double)i * i;
        b += 2.0;
        d = 1.0 / (a * d + b);
        c = b + a / c;
        const double del = c * d;
        h *= del;
        if (std::fabs(del - 1.0) < 1e-16) break;
    }
    return h * std::exp(-x);
}

// Maxwellian-averaged Lotz rate, m^3/s
double lotz_rate(double P_eV, int q, double Te_eV)
{
    const double x = P_eV / Te_eV;
    if (x > 700.0) return 0.0;
    return std::sqrt(8.0 * kE / (kPi * kMe)) * kLotzA * q * expint_e1(x) / (x * std::pow(Te_eV, 1.5));
}

// Nanbu's A(s): root of coth(A) - 1/A = exp(-s), by bisection on ln A in FP64.
// L(A) = coth A - 1/A is evaluated from its series for small A.
double nanbu_A_host(double s)
{
    const double y = std::exp(-s);
    auto L = [](double A) {
        if (A < 1e-3) return A / 3.0 - A * A * A / 45.0;
        return 1.0 / std::tanh(A) - 1.0 / A;
    };
    double lo = std::log(1e-12), hi = std::log(2.0 / (-std::expm1(-s)) + 10.0);
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (L(std::exp(mid)) < y) lo = mid; else hi = mid;
    }
    return std::exp(0.5 * (lo + hi));
}

struct HostRun {
    ecris_geometry geo;
    ecris_bfield bf;
    int nx, ny, nz;
    double ne_in, ne_out, Te_w, Te_c;
    double mass_amu;
    int qmax;
    std::vector<double> ip;
    std::vector<int> nout;
    std::vector<double> rate[2];   // m^3/s per Q, zone 0 cold, 1 warm
    std::vector<double> rate2[2];  // double ionisation Q -> Q+2 (m^3/s), same layout
    std::vector<double> rate3[2];  // triple ionisation Q -> Q+3 (m^3/s), same layout
    std::vector<double> rate_r[2]; // recombination Q -> Q-1 (m^3/s), Q = 0..qmax
    float ne_max[2] = {0.f, 0.f};  // largest FP32 n_e (as the kernels see it) of the cold and warm cells
    std::vector<unsigned char> cell_zone;
    ecris_mcc mcc;
    double zm;
    bool has_e = false;            // some cell of the E grid is nonzero
    std::vector<double> bmag;      // |B| at the cell centres (T)
    std::vector<double> ax_y, ax_M;   // on-axis table and its spline's second derivatives (empty: mirror)
    uint64_t steps_mark = 0;       // steps at the last n_e update (or load)
};

// Natural cubic spline through n samples at z_k = k h: second derivatives
// M_0 = M_{n-1} = 0 and M_{k-1} + 4 M_k + M_{k+1} = 6 (y_{k+1} - 2 y_k +
// y_{k-1}) / h^2 for the inner points (tridiagonal elimination)
void axial_spline(const std::vector<double>& y, double L, std::vector<double>& M)
{
    const size_t n = y.size();
    const double h = L / (double)(n - 1);
    M.assign(n, 0.0);
    std::vector<double> cp(n, 0.0), dp(n, 0.0);
    for (size_t k = 1; k + 1 < n; ++k) {
        const double r = 6.0 * (y[k + 1] - 2.0 * y[k] + y[k - 1]) / (h * h);
        const double m = 4.0 - cp[k - 1];
        cp[k] = 1.0 / m;
        dp[k] = (r - dp[k - 1]) / m;
    }
    for (size_t k = n - 2; k >= 1; --k) {
        M[k] = dp[k] - cp[k] * M[k + 1];
        if (k == 1) break;
    }
}

// on-axis B0 and its first two derivatives: the table's spline, or the
// synthetic mirror
void b0_host(const HostRun& h, double z, double& b0, double& b1, double& b2)
{
    if (!h.ax_y.empty()) {
        const size_t n = h.ax_y.size();
        const double hz = h.geo.L / (double)(n - 1);
        long k = (long)std::floor(z / hz);
        k = k < 0 ? 0 : (k > (long)n - 2 ? (long)n - 2 : k);
        const double t = z / hz - (double)k, u = 1.0 - t;
        const double y0 = h.ax_y[k], y1 = h.ax_y[k + 1], m0 = h.ax_M[k], m1 = h.ax_M[k + 1];
        b0 = u * y0 + t * y1 + hz * hz / 6.0 * ((u * u * u - u) * m0 + (t * t * t - t) * m1);
        b1 = (y1 - y0) / hz + hz / 6.0 * ((3.0 * t * t - 1.0) * m1 - (3.0 * u * u - 1.0) * m0);
        b2 = u * m0 + t * m1;
        return;
    }
    const double bmin = h.bf.B_min;
    if (z <= h.zm) {
        const double a = 0.5 * (h.bf.B_inj - bmin), k = kPi / h.zm;
        b0 = bmin + a * (1.0 + std::cos(k * z));
        b1 = -a * k * std::sin(k * z);
        b2 = -a * k * k * std::cos(k * z);
    } else {
        const double a = 0.5 * (h.bf.B_ext - bmin), k = kPi / (h.geo.L - h.zm);
        b0 = bmin + a * (1.0 - std::cos(k * (z - h.zm)));
        b1 = a * k * std::sin(k * (z - h.zm));
        b2 = a * k * k * std::cos(k * (z - h.zm));
    }
}

uint32_t float_bits(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, sizeof u);
    return u;
}

// The ionisation word above which no cell can ionise an atom: the kernels'
// FP32 product n_e k_0 dt, largest over the cells (the largest n_e of each
// zone times its k_0 dt), with a relative margin of 1e-4 that covers any
// rounding difference in the probability, as ceil((1 - exp(-lambda)) 2^32);
// never 0, which the kernels read as "take the device's word"
uint32_t atom_gate_host(const float ne_max[2], const float* kdt)
{
    const float lam = std::max(ne_max[0] * kdt[0], ne_max[1] * kdt[kQSlots]);
    const float lam_max = lam * 1.0001f;
    const double pmax = -std::expm1(-(double)lam_max);
    const double gate = std::ceil(pmax * 4294967296.0);
    if (gate >= 4294967295.0) return 0xFFFFFFFFu;
    return gate < 1.0 ? 1u : (uint32_t)gate;
}

double bmag_host(const HostRun& h, double x, double y, double z)
{
    double b0, b1, b2;
    b0_host(h, z, b0, b1, b2);
    const double hc = h.bf.B_hex / (h.geo.R0 * h.geo.R0);
    const double Bx = -0.5 * x * b1 + hc * 2.0 * x * y;
    const double By = -0.5 * y * b1 + hc * (x * x - y * y);
    const double Bz = b0 - 0.25 * (x * x + y * y) * b2;
    return std::sqrt(Bx * Bx + By * By + Bz * Bz);
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

}  // namespace

void ecris::ecris_internal_set_thread_error(const char* msg) { g_create_error = msg; }

namespace {

enum { kKindStep = 0, kKindCoulomb = 1, kKindOther = 2 };

// kernel timing (ecris_set_profiling / ecris_batch_set_profiling): launches
// bracketed by events on the launching stream, read back when collected
struct KernelTimer {
    bool on = false;
    struct Timed { int kind; int kernels; cudaEvent_t a, b; };
    std::vector<Timed> pending;
    std::vector<cudaEvent_t> pool;
    int64_t launches[3] = {0, 0, 0};
    double ms[3] = {0.0, 0.0, 0.0};

    cudaEvent_t take()
    {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }

    template <class F>
    cudaError_t run(int kind, cudaStream_t s, F fn, int kernels = 1)
    {
        if (!on) return fn();
        cudaEvent_t a = take(), b = take();
        if (!a || !b) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaEventRecord(a, s);
        if (e == cudaSuccess) e = fn();
        if (e == cudaSuccess) e = cudaEventRecord(b, s);
        pending.push_back({kind, kernels, a, b});
        return e;
    }

    cudaError_t collect(cudaStream_t s)
    {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        for (auto& t : pending) {
            float m = 0.0f;
            e = cudaEventElapsedTime(&m, t.a, t.b);
            if (e != cudaSuccess) return e;
            launches[t.kind] += t.kernels;
            ms[t.kind] += m;
            pool.push_back(t.a);
            pool.push_back(t.b);
        }
        pending.clear();
        return cudaSuccess;
    }

    void reset(bool enable)
    {
        on = enable;
        for (int k = 0; k < 3; ++k) {
            launches[k] = 0;
            ms[k] = 0.0;
        }
    }

    void fill(ecris_profile* out) const
    {
        out->step_launches = launches[kKindStep];
        out->step_ms = ms[kKindStep];
        out->coulomb_launches = launches[kKindCoulomb];
        out->coulomb_ms = ms[kKindCoulomb];
        out->other_launches = launches[kKindOther];
        out->other_ms = ms[kKindOther];
    }

    void release()
    {
        for (auto& t : pending) {
            cudaEventDestroy(t.a);
            cudaEventDestroy(t.b);
        }
        pending.clear();
        for (auto e : pool) cudaEventDestroy(e);
        pool.clear();
    }
};

}  // namespace

constexpr uint32_t kSortAfterLoad = 8;   // steps of one ecris_step call that sort a fresh load first

// what a captured step graph bakes in: the parameter block (by value) and
// the launch shapes
struct GraphKey {
    RunDev R;
    uint32_t ntiles;
    int step_grid, collide_grid;
};

struct ecris_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sm_count = 0;
    int step_grid = 0;
    std::string err;
    bool failed = false;

    bool have_fields = false;
    HostRun h;
    float4* d_cell = nullptr;
    double* d_rlc = nullptr;        // 2.38e-6 sqrt(T_e)/(B dX) per cell: R_L n_e of the delta stencil
    bool ne_device = false;         // n_e was updated on the device: the host no longer knows its maxima
    float4* d_E = nullptr;
    float* d_kdt = nullptr;
    float4* d_btab = nullptr;       // on-axis table, one cubic per segment
    float* d_nanbu = nullptr;

    bool have_ions = false;     // device buffers allocated
    bool loaded = false;        // a valid ensemble is loaded
    size_t cap = 0, cap_cells = 0;
    size_t n = 0, n4 = 0;
    uint8_t* d_q8 = nullptr;
    unsigned int* d_bad = nullptr;
    uint32_t* d_err = nullptr;
    uint4* d_plist = nullptr;
    float4* d_pvel = nullptr;
    uint32_t* d_tcount = nullptr;
    float4* d_crec = nullptr;
    uint32_t* d_ccount = nullptr;
    uint32_t* d_cstart = nullptr;
    uint32_t* d_crange = nullptr;   // collision ranges: size this step, largest cell count seen
    uint32_t* d_coff = nullptr;
    unsigned long long* d_cstat = nullptr;   // scan tile status words and ticket counter
    unsigned long long* d_ckeys = nullptr;
    int collide_grid = 0;
    // two sets of particle arrays; the sort moves the particles from the
    // current set (index cur) to the other
    float* d_soa[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    uint32_t* d_meta = nullptr;
    uint32_t* d_id = nullptr;
    float* d_soa2[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    uint32_t* d_meta2 = nullptr;
    uint32_t* d_id2 = nullptr;
    uint32_t* d_hist = nullptr;    // sort histogram (2 Nc + 1), kept zero between sorts
    uint32_t* d_hoff = nullptr;    // its exclusive scan (2 Nc + 2)
    uint32_t* d_hblk = nullptr;    // scan block totals
    uint32_t sort_every = 32;      // steps between sorts
    uint32_t since_sort = 0;
    bool fresh = false;         // loaded, not yet sorted
    uint32_t calls_since_load = 0;
    int parity = 0;                // which particle set is current (flips at each sort)
    // captured per-step kernel sequences, by particle set and kind (0: the
    // whole step, 1: the collision kernels only), each valid for the launch
    // arguments it was captured with (a reload into the same buffers with
    // the same step length keeps them, so a load-step-read cycle does not
    // re-instantiate its graph)
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    GraphKey gkey[2][2];
    uint32_t* d_cslot = nullptr;
    uint32_t* d_sslot = nullptr;
    unsigned long long* d_dep = nullptr;
    unsigned long long* d_count = nullptr;
    unsigned long long* d_charge = nullptr;
    unsigned long long* d_mark = nullptr;   // d_charge at the last n_e update (or load)
    double* d_ne64 = nullptr;               // scratch of the n_e update: FP64 n_e per cell
    unsigned long long* d_tally = nullptr;
    unsigned long long* d_census = nullptr;
    uint32_t* d_step = nullptr;
    uint32_t* d_leave = nullptr;    // leaver list (cap) and its count
    uint32_t* d_birth = nullptr;    // ionisation step by particle id (cap)
    // moment probes and screens
    int32_t* d_pslot = nullptr;     // per cell: probe slot or -1
    double* d_pmom = nullptr;       // [slot][qmax + 1][7]
    unsigned long long* d_pscreen = nullptr;   // [screen][qmax + 1][pixels^2]
    size_t probe_cells = 0;
    size_t screen_words = 0;
    ProbeDev probe{};
    bool have_probes = false;
    uint64_t probe_samples = 0;
    unsigned long long* d_fptd = nullptr;   // first-passage histogram and age sums
    uint32_t* d_nleave = nullptr;
    unsigned int* d_ticket = nullptr;
    uint32_t ntiles = 0;
    uint32_t tile = kTile;      // particles per tile of the step kernel (a batch sets its launch shape's)
    uint32_t btiles = 0;        // tiles of the run in its batch's launch shape
    RunDev* h_run = nullptr;    // parameter block passed by value to every kernel
    float* h_kdt = nullptr;     // pinned staging copy of the rate table
    double weight = 0.0;
    uint64_t seed = 0;
    uint64_t steps_done = 0;
    double time_s = 0.0;
    double dt_loaded = -1.0;
    uint32_t fold_every = 1, since_fold = 0;

    KernelTimer timer;          // ecris_set_profiling
};

namespace {

ecris_status fail(ecris_ctx* c, ecris_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
    return st;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            ctx->failed = true;                                                           \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? ECRIS_ENOMEM : ECRIS_ECUDA, \
                        "%s: %s", #call, cudaGetErrorString(e_));                         \
        }                                                                                 \
    } while (0)

// launch `fn` on the context stream; with profiling on, bracket it by events
template <class F>
cudaError_t timed(ecris_ctx* ctx, int kind, F fn, int kernels = 1)
{
    return ctx->timer.run(kind, ctx->stream, fn, kernels);
}

template <class T>
void free_async(ecris_ctx* ctx, T*& p)
{
    if (p) cudaFreeAsync(p, ctx->stream);
    p = nullptr;
}

void free_graphs(ecris_ctx* ctx)
{
    for (auto& row : ctx->gexec)
        for (auto& x : row) {
            if (x) cudaGraphExecDestroy(x);
            x = nullptr;
        }
}

void free_ions(ecris_ctx* ctx)
{
    free_graphs(ctx);
    for (auto& p : ctx->d_soa) free_async(ctx, p);
    free_async(ctx, ctx->d_meta);
    free_async(ctx, ctx->d_id);
    for (auto& p : ctx->d_soa2) free_async(ctx, p);
    free_async(ctx, ctx->d_meta2);
    free_async(ctx, ctx->d_id2);
    free_async(ctx, ctx->d_hist);
    free_async(ctx, ctx->d_hoff);
    free_async(ctx, ctx->d_hblk);
    free_async(ctx, ctx->d_cslot);
    free_async(ctx, ctx->d_sslot);
    free_async(ctx, ctx->d_dep);
    free_async(ctx, ctx->d_count);
    free_async(ctx, ctx->d_charge);
    free_async(ctx, ctx->d_mark);
    free_async(ctx, ctx->d_ne64);
    free_async(ctx, ctx->d_tally);
    free_async(ctx, ctx->d_census);
    free_async(ctx, ctx->d_step);
    free_async(ctx, ctx->d_leave);
    free_async(ctx, ctx->d_birth);
    free_async(ctx, ctx->d_fptd);
    free_async(ctx, ctx->d_nleave);
    free_async(ctx, ctx->d_ticket);
    free_async(ctx, ctx->d_q8);
    free_async(ctx, ctx->d_bad);
    free_async(ctx, ctx->d_err);
    free_async(ctx, ctx->d_plist);
    free_async(ctx, ctx->d_pvel);
    free_async(ctx, ctx->d_tcount);
    free_async(ctx, ctx->d_crec);
    free_async(ctx, ctx->d_ccount);
    free_async(ctx, ctx->d_cstart);
    free_async(ctx, ctx->d_crange);
    free_async(ctx, ctx->d_coff);
    free_async(ctx, ctx->d_cstat);
    free_async(ctx, ctx->d_ckeys);
    ctx->have_ions = false;
    ctx->loaded = false;
    ctx->cap = ctx->cap_cells = 0;
}

void free_fields(ecris_ctx* ctx)
{
    free_async(ctx, ctx->d_cell);
    free_async(ctx, ctx->d_rlc);
    free_async(ctx, ctx->d_E);
    free_async(ctx, ctx->d_kdt);
    free_async(ctx, ctx->d_btab);
    free_async(ctx, ctx->d_nanbu);
    free_async(ctx, ctx->d_pslot);
    free_async(ctx, ctx->d_pmom);
    free_async(ctx, ctx->d_pscreen);
    ctx->have_probes = false;
    ctx->have_fields = false;
}

// zero the probes' sums (after installing them, and at every load)
ecris_status zero_probes(ecris_ctx* ctx)
{
    if (!ctx->have_probes) return ECRIS_OK;
    const size_t qs = (size_t)ctx->h.qmax + 1;
    if (ctx->probe_cells)
        CK(cudaMemsetAsync(ctx->d_pmom, 0, ctx->probe_cells * qs * 7 * sizeof(double), ctx->stream));
    if (ctx->screen_words)
        CK(cudaMemsetAsync(ctx->d_pscreen, 0, ctx->screen_words * sizeof(unsigned long long), ctx->stream));
    ctx->probe_samples = 0;
    return ECRIS_OK;
}

// FP32 kernel constants of the run for time step dt (built in FP64)
void fill_rundev(ecris_ctx* ctx, double dt, RunDev& R)
{
    const HostRun& h = ctx->h;
    const double M = h.mass_amu * kAmu;
    std::memset(&R, 0, sizeof R);
    R.R0 = (float)h.geo.R0;
    R.R0sq = (float)(h.geo.R0 * h.geo.R0);
    R.L = (float)h.geo.L;
    R.r_ap_sq = (float)(h.geo.r_ap * h.geo.r_ap);
    R.eps_wall = (float)(1e-6 * h.geo.L);
    R.inlet_x = (float)h.geo.inlet[0];
    R.inlet_y = (float)h.geo.inlet[1];
    R.inlet_z = (float)h.geo.inlet[2];
    R.B_min = (float)h.bf.B_min;
    const double aL = 0.5 * (h.bf.B_inj - h.bf.B_min), aR = 0.5 * (h.bf.B_ext - h.bf.B_min);
    const double kL = kPi / h.zm, kR = kPi / (h.geo.L - h.zm);
    R.aL = (float)aL;
    R.aR = (float)aR;
    R.zm = (float)h.zm;
    R.inv_zm = (float)(1.0 / h.zm);
    R.inv_zr = (float)(1.0 / (h.geo.L - h.zm));
    R.aLk = (float)(aL * kL);
    R.aLk2 = (float)(aL * kL * kL);
    R.aRk = (float)(aR * kR);
    R.aRk2 = (float)(aR * kR * kR);
    R.hex_c = (float)(h.bf.B_hex / (h.geo.R0 * h.geo.R0));
    R.B_ecr = (float)h.bf.B_ecr;
    R.nx = h.nx;
    R.ny = h.ny;
    R.nz = h.nz;
    const double dx = 2.0 * h.geo.R0 / h.nx, dy = 2.0 * h.geo.R0 / h.ny, dz = h.geo.L / h.nz;
    R.inv_dx = (float)(1.0 / dx);
    R.inv_dy = (float)(1.0 / dy);
    R.inv_dz = (float)(1.0 / dz);
    R.qmax = h.qmax;
    R.qm_unit = (float)(kE / M);
    R.dt = (float)dt;
    R.half_dt = (float)(0.5 * dt);
    R.flags = (h.mcc.flags & ~kFHasE) | (h.has_e ? kFHasE : 0u);
    R.sig0 = (float)std::sqrt(h.mcc.T0_eV * kE / M);
    R.n0s1 = (float)(h.mcc.n0_cm3 * 1e6 * h.mcc.sigma1_cm2 * 1e-4);
    R.vth2 = (float)(8.0 * h.mcc.T0_eV * kE / (kPi * M));
    R.dv_cx = (float)std::sqrt(2.0 * 0.5 * h.mcc.E_cx_eV * kE / M);
    R.n0sel = (h.mcc.flags & kFElastic) ? (float)(h.mcc.n0_cm3 * 1e6 * h.mcc.sigma_el1_cm2 * 1e-4) : 0.0f;
    R.sig_refl = h.mcc.T_refl_eV > 0.0 ? (float)std::sqrt(h.mcc.T_refl_eV * kE / M) : R.sig0;
    for (int zone = 0; zone < 2; ++zone) {
        const double Te = zone ? h.Te_w : h.Te_c;
        R.ei_coef[zone] = (float)(3.715e-6 * h.mcc.lnL_ei * dt / (h.mass_amu * h.mass_amu * std::sqrt(Te)));
    }
    R.ei_pow = h.mcc.ei_charge_power;
    R.ke_scale = (float)(0.5 * M / kE * 1e6);
    R.lnl_ii_coef = coulomb_s_coef(h.mcc.lnL_ii, h.mass_amu, ctx->weight, dx * dy * dz);
    R.seed_lo = (uint32_t)ctx->seed;
    R.seed_hi = (uint32_t)(ctx->seed >> 32);
    R.x = reinterpret_cast<int32_t*>(ctx->d_soa[0]);
    R.y = reinterpret_cast<int32_t*>(ctx->d_soa[1]);
    R.z = reinterpret_cast<int32_t*>(ctx->d_soa[2]);
    R.sxy = (float)(h.geo.R0 / 2147483648.0);
    R.inv_sxy = (float)(2147483648.0 / h.geo.R0);
    R.sz = (float)(h.geo.L / 4294967296.0);
    R.inv_sz = (float)(4294967296.0 / h.geo.L);
    R.dt_sxy = (float)(dt * 2147483648.0 / h.geo.R0);
    R.dt_sz = (float)(dt * 4294967296.0 / h.geo.L);
    R.R0_d = h.geo.R0;
    R.L_d = h.geo.L;
    R.r_ap_d = h.geo.r_ap;
    R.eps_wall_d = 1e-6 * h.geo.L;
    R.sxy_d = h.geo.R0 / 2147483648.0;
    R.sz_d = h.geo.L / 4294967296.0;
    R.inlet_X = (int32_t)std::llrint(h.geo.inlet[0] / R.sxy_d);
    R.inlet_Y = (int32_t)std::llrint(h.geo.inlet[1] / R.sxy_d);
    R.inlet_Z = (int32_t)(std::llrint(h.geo.inlet[2] / R.sz_d) - 2147483648ll);
    R.vx = ctx->d_soa[3];
    R.vy = ctx->d_soa[4];
    R.vz = ctx->d_soa[5];
    R.meta = ctx->d_meta;
    R.id = ctx->d_id;
    R.cell = ctx->d_cell;
    R.E = ctx->d_E;
    R.kdt = ctx->d_kdt;
    R.btab = ctx->d_btab;
    R.nseg = ctx->h.ax_y.empty() ? 0 : (int32_t)ctx->h.ax_y.size() - 1;
    R.inv_h = ctx->h.ax_y.empty() ? 0.0f : (float)((double)R.nseg / ctx->h.geo.L);
    R.dep = ctx->d_dep;
    R.tally = ctx->d_tally;
    R.plist = ctx->d_plist;
    R.pvel = ctx->d_pvel;
    R.tcount = ctx->d_tcount;
    R.crec = ctx->d_crec;
    R.ccount = ctx->d_ccount;
    R.cstart = ctx->d_cstart;
    R.crange = ctx->d_crange;
    R.coff = ctx->d_coff;
    R.cstat = ctx->d_cstat;
    R.cctr = ctx->d_cstat ? ctx->d_cstat + coulomb_scan_blocks((uint32_t)ctx->cap_cells) : nullptr;
    R.ckeys = ctx->d_ckeys;
    R.cslot = ctx->d_cslot;
    R.sslot = ctx->d_sslot;
    R.nanbu = ctx->d_nanbu;
    R.nanbu_lnlo = (float)std::log(kNanbuSLo);
    R.nanbu_inv_dln = (float)((kNanbuN - 1) / std::log(kNanbuSHi / kNanbuSLo));
    R.step = ctx->d_step;
    R.err = ctx->d_err;
    R.leave = ctx->d_leave;
    R.birth = ctx->d_birth;
    R.fptd = ctx->d_fptd;
    R.nleave = ctx->d_nleave;
    R.n = (uint32_t)ctx->n;
    R.n4 = (uint32_t)ctx->n4;
    R.ncells = (uint32_t)((size_t)h.nx * h.ny * h.nz);
    R.tile = ctx->tile;
}

// The per-cell records the kernels read, {n_e, zone, delta_x, delta_y}, from
// n_e (m^-3) and the zone flags, in FP64: delta follows the printed stencil
// (y-differences for delta_x, x-differences for delta_y) scaled by
// R_L = 2.38e-6 sqrt(T_e) / (B dX) / n_e; neighbours outside the mesh take the
// edge value and a cell with n_e = 0 gets delta = 0 (Sec. II).
void cell_records(HostRun& h, const std::vector<double>& ne, const std::vector<unsigned char>& zone,
                  std::vector<float4>& cell)
{
    const size_t nc = (size_t)h.nx * h.ny * h.nz;
    const double dx = 2.0 * h.geo.R0 / h.nx;
    cell.assign(nc, make_float4(0.f, 0.f, 0.f, 0.f));
    h.ne_max[0] = h.ne_max[1] = 0.0f;
    h.cell_zone.assign(nc, 0);
    auto NE = [&](int iz, int iy, int ix) {
        iy = iy < 0 ? 0 : (iy >= h.ny ? h.ny - 1 : iy);
        ix = ix < 0 ? 0 : (ix >= h.nx ? h.nx - 1 : ix);
        return ne[((size_t)iz * h.ny + iy) * h.nx + ix];
    };
    for (int iz = 0; iz < h.nz; ++iz)
        for (int iy = 0; iy < h.ny; ++iy)
            for (int ix = 0; ix < h.nx; ++ix) {
                const size_t c = ((size_t)iz * h.ny + iy) * h.nx + ix;
                double dlx = 0.0, dly = 0.0;
                // isotropic heating (Sec. IV): no drift bias
                if (ne[c] > 0.0 && !(h.mcc.flags & kFIsoheat)) {
                    const double Te = zone[c] ? h.Te_w : h.Te_c;
                    const double rl = 2.38e-6 * std::sqrt(Te) / (h.bmag[c] * dx) / ne[c];
                    const double sx = NE(iz, iy - 1, ix) - NE(iz, iy + 1, ix) +
                                      0.5 * (NE(iz, iy - 1, ix + 1) + NE(iz, iy - 1, ix - 1) -
                                             NE(iz, iy + 1, ix - 1) - NE(iz, iy + 1, ix + 1));
                    const double sy = NE(iz, iy, ix + 1) - NE(iz, iy, ix - 1) +
                                      0.5 * (NE(iz, iy + 1, ix + 1) + NE(iz, iy - 1, ix + 1) -
                                             NE(iz, iy + 1, ix - 1) - NE(iz, iy - 1, ix - 1));
                    dlx = -rl * sx;
                    dly = -rl * sy;
                }
                cell[c] = make_float4((float)ne[c], zone[c] ? 1.0f : 0.0f, (float)dlx, (float)dly);
                float& m = h.ne_max[zone[c] ? 1 : 0];
                if (cell[c].x > m) m = cell[c].x;
                h.cell_zone[c] = zone[c];
            }
}

// upload the parameter block and rate table for step length dt
ecris_status upload_dt(ecris_ctx* ctx, double dt)
{
    if (dt == ctx->dt_loaded) return ECRIS_OK;
    // the pinned staging buffers may still feed an earlier copy
    CK(cudaStreamSynchronize(ctx->stream));
    fill_rundev(ctx, dt, *ctx->h_run);
    // k dt with k = k1 (+ k2 with double ionisation, + kr with
    // recombination), and the shares k1 / k and (k1 + k2) / k
    const uint32_t fl = ctx->h.mcc.flags;
    const bool dbl = (fl & kFDouble) != 0, rec = (fl & kFRecomb) != 0;
    for (int zone = 0; zone < 2; ++zone)
        for (int q = 0; q < kQSlots; ++q) {
            // with recombination on the variant kernel reads these for every
            // ion, so ionisation enters only where it is switched on
            const bool ion = q < ctx->h.qmax && (!rec || (fl & kFIonize));
            const double k1 = ion ? ctx->h.rate[zone][q] : 0.0;
            const double k2 = (dbl && ion) ? ctx->h.rate2[zone][q] : 0.0;
            const double k3 = (dbl && ion) ? ctx->h.rate3[zone][q] : 0.0;
            const double kr = (rec && q <= ctx->h.qmax) ? ctx->h.rate_r[zone][q] : 0.0;
            const double k = k1 + k2 + k3 + kr;
            ctx->h_kdt[zone * kQSlots + q] = (float)(k * dt);
            ctx->h_kdt[2 * kQSlots + zone * kQSlots + q] = k > 0.0 ? (float)(k1 / k) : 1.0f;
            ctx->h_kdt[4 * kQSlots + zone * kQSlots + q] = k > 0.0 ? (float)((k1 + k2) / k) : 1.0f;
            ctx->h_kdt[6 * kQSlots + zone * kQSlots + q] = k > 0.0 ? (float)((k1 + k2 + k3) / k) : 1.0f;
        }
    CK(cudaMemcpyAsync(ctx->d_kdt, ctx->h_kdt, kGateWord * sizeof(float), cudaMemcpyHostToDevice,
                       ctx->stream));
    // the atom gate on the device, from the new k_0 dt and the largest n_e of
    // each zone that the device keeps (a device update of n_e changes them),
    // and by value in the parameter block while the host knows those maxima.
    // Rounding to nearest is monotone, so over the cells of one zone the
    // largest FP32 product n_e k_0 dt is the product of the largest n_e
    CK(launch_atom_gate(ctx->d_kdt, ctx->stream));
    ctx->h_run->atom_gate = ctx->ne_device ? 0u : atom_gate_host(ctx->h.ne_max, ctx->h_kdt);
    ctx->dt_loaded = dt;
    return ECRIS_OK;
}

// Self-consistent electron density (Sec. II: n_e equals the ion charge
// density, by charge neutrality).  Folds the deposit, takes the charge each
// cell received since the last update (or the load), time-averages it over
// the steps in between, n_e = w sum(Q) / (steps V_cell), and rebuilds every
// cell's {n_e, zone, delta} record and the atom gate from it (Sec. II, the
// delta stencil and R_L of the heating kick).  The zones stay (they follow
// |B|).  All of it runs on the device in stream order after the queued
// steps: nothing is read back and the host does not wait.
ecris_status update_ne(ecris_ctx* ctx)
{
    HostRun& h = ctx->h;
    if (ctx->steps_done <= h.steps_mark)
        return fail(ctx, ECRIS_ESTATE, "update_ne: no step since the load or the last update");
    const uint32_t nc = (uint32_t)((size_t)h.nx * h.ny * h.nz);
    if (ctx->dt_loaded < 0.0) {
        ecris_status st = upload_dt(ctx, 1e-9);   // parameter block for the fold kernel
        if (st != ECRIS_OK) return st;
    }
    CK(launch_fold(*ctx->h_run, nc, ctx->d_count, ctx->d_charge, ctx->stream));
    ctx->since_fold = 0;
    const double vol = (2.0 * h.geo.R0 / h.nx) * (2.0 * h.geo.R0 / h.ny) * (h.geo.L / h.nz);
    const double steps = (double)(ctx->steps_done - h.steps_mark);
    CK(launch_ne_update(ctx->d_charge, ctx->d_mark, ctx->d_ne64, ctx->d_rlc, ctx->d_cell, ctx->d_kdt, h.nx, h.ny,
                        nc, ctx->weight, steps * vol, (h.mcc.flags & kFIsoheat) != 0, ctx->sm_count, ctx->stream));
    h.steps_mark = ctx->steps_done;
    // the gate now lives on the device (k_atom_gate ran with the update)
    ctx->ne_device = true;
    ctx->h_run->atom_gate = 0u;
    return ECRIS_OK;
}

ecris_status get_fptd(ecris_ctx* ctx, uint64_t* hist, uint64_t* age_sum)
{
    std::vector<unsigned long long> f(kFptdWords);
    CK(cudaMemcpyAsync(f.data(), ctx->d_fptd, kFptdWords * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int q = 0; q <= ctx->h.qmax; ++q) {
        if (hist)
            for (int b = 0; b < kFptdBins; ++b) hist[(size_t)q * kFptdBins + b] = f[(size_t)q * kFptdBins + b];
        if (age_sum) age_sum[q] = f[(size_t)kFptdAgeSum + q];
    }
    return ECRIS_OK;
}

ecris_status get_extraction_radius(ecris_ctx* ctx, double* r_sum)
{
    std::vector<unsigned long long> f(kQSlots);
    CK(cudaMemcpyAsync(f.data(), ctx->d_fptd + kFptdRadius, kQSlots * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int q = 0; q <= ctx->h.qmax; ++q) r_sum[q] = (double)f[q] * 1e-9;
    return ECRIS_OK;
}

ecris_status set_probes(ecris_ctx* ctx, const ecris_probe_spec* sp)
{
    const HostRun& h = ctx->h;
    const size_t nc = (size_t)h.nx * h.ny * h.nz;
    if (sp->ncells > nc || (sp->ncells && !sp->cells))
        return fail(ctx, ECRIS_EINVAL, "set_probes: need ncells <= Nc and a cell list");
    if (sp->nscreens < 0 || sp->nscreens > kMaxScreens)
        return fail(ctx, ECRIS_EINVAL, "set_probes: 0 <= nscreens <= %d", kMaxScreens);
    std::vector<int32_t> slot(nc, -1);
    for (size_t k = 0; k < sp->ncells; ++k) {
        const uint32_t c = sp->cells[k];
        if (c >= nc) return fail(ctx, ECRIS_EINVAL, "set_probes: cell %u out of range", c);
        if (slot[c] >= 0) return fail(ctx, ECRIS_EINVAL, "set_probes: cell %u listed twice", c);
        slot[c] = (int32_t)k;
    }
    ProbeDev P{};
    P.qs = h.qmax + 1;
    P.nscreens = sp->nscreens;
    if (sp->nscreens) {
        int lg = 0;
        while ((1 << lg) < sp->pixels && lg < 13) ++lg;
        if (sp->pixels < 2 || sp->pixels > 4096 || (1 << lg) != sp->pixels)
            return fail(ctx, ECRIS_EINVAL, "set_probes: pixels must be a power of two in [2, 4096]");
        P.pix_log2 = lg;
        // z = U L / 2^32 for U = Z + 2^31: the slab z_lo <= z < z_hi is
        // ceil(z_lo 2^32 / L) <= U <= ceil(z_hi 2^32 / L) - 1
        const double per = 4294967296.0 / h.geo.L;
        for (int k = 0; k < sp->nscreens; ++k) {
            const double lo = sp->z_lo[k], hi = sp->z_hi[k];
            if (!std::isfinite(lo) || !std::isfinite(hi) || !(lo >= 0.0) || !(hi > lo) || hi > h.geo.L)
                return fail(ctx, ECRIS_EINVAL, "set_probes: screen %d needs 0 <= z_lo < z_hi <= L", k);
            const double ulo = std::ceil(lo * per), uhi = std::ceil(hi * per) - 1.0;
            P.ulo[k] = (uint32_t)std::min(ulo, 4294967295.0);
            P.uhi[k] = (uint32_t)std::max(0.0, std::min(uhi, 4294967295.0));
        }
    }
    const size_t words = (size_t)sp->nscreens * P.qs << (2 * P.pix_log2);
    if (words * sizeof(unsigned long long) > ((size_t)16 << 30))
        return fail(ctx, ECRIS_EINVAL, "set_probes: screens above 16 GB");
    CK(cudaSetDevice(ctx->device));
    free_async(ctx, ctx->d_pslot);
    free_async(ctx, ctx->d_pmom);
    free_async(ctx, ctx->d_pscreen);
    ctx->have_probes = false;
    if (sp->ncells) {
        CK(cudaMallocAsync((void**)&ctx->d_pslot, nc * sizeof(int32_t), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_pmom, sp->ncells * P.qs * 7 * sizeof(double), ctx->stream));
        CK(cudaMemcpyAsync(ctx->d_pslot, slot.data(), nc * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    }
    if (words) CK(cudaMallocAsync((void**)&ctx->d_pscreen, words * sizeof(unsigned long long), ctx->stream));
    P.slot = ctx->d_pslot;
    P.mom = ctx->d_pmom;
    P.screen = ctx->d_pscreen;
    ctx->probe = P;
    ctx->probe_cells = sp->ncells;
    ctx->screen_words = words;
    ctx->have_probes = true;
    ecris_status st = zero_probes(ctx);
    CK(cudaStreamSynchronize(ctx->stream));   // the slot map's host copy dies at return
    return st;
}

ecris_status probe_sample(ecris_ctx* ctx)
{
    if (!ctx->have_probes) return fail(ctx, ECRIS_ESTATE, "probe_sample: call ecris_set_probes first");
    if (ctx->dt_loaded < 0.0) {
        ecris_status st = upload_dt(ctx, 1e-9);   // parameter block for the probe kernel
        if (st != ECRIS_OK) return st;
    }
    CK(launch_probe(*ctx->h_run, ctx->probe, (uint32_t)ctx->n4, ctx->sm_count, ctx->stream));
    ++ctx->probe_samples;
    return ECRIS_OK;
}

ecris_status get_probes(ecris_ctx* ctx, uint64_t* samples, double* moments, uint64_t* screens)
{
    if (!ctx->have_probes) return fail(ctx, ECRIS_ESTATE, "get_probes: call ecris_set_probes first");
    const size_t qs = (size_t)ctx->h.qmax + 1;
    if (moments && ctx->probe_cells)
        CK(cudaMemcpyAsync(moments, ctx->d_pmom, ctx->probe_cells * qs * 7 * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->stream));
    if (screens && ctx->screen_words)
        CK(cudaMemcpyAsync(screens, ctx->d_pscreen, ctx->screen_words * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (samples) *samples = ctx->probe_samples;
    return ECRIS_OK;
}

ecris_status get_cells(ecris_ctx* ctx, float* ne, float* delta_x, float* delta_y)
{
    const size_t nc = (size_t)ctx->h.nx * ctx->h.ny * ctx->h.nz;
    std::vector<float4> cell(nc);
    CK(cudaMemcpyAsync(cell.data(), ctx->d_cell, nc * sizeof(float4), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (size_t c = 0; c < nc; ++c) {
        if (ne) ne[c] = cell[c].x;
        if (delta_x) delta_x[c] = cell[c].z;
        if (delta_y) delta_y[c] = cell[c].w;
    }
    return ECRIS_OK;
}

// the kernel sequence of one step, captured once per particle set and
// parameter block and replayed as a CUDA graph
ecris_status step_graph(ecris_ctx* ctx, int kind, cudaGraphExec_t* out)
{
    const int p = ctx->parity;
    GraphKey key;
    std::memset(&key, 0, sizeof key);
    std::memcpy(&key.R, ctx->h_run, sizeof(RunDev));   // the block was zeroed before it was filled
    key.ntiles = ctx->ntiles;
    key.step_grid = ctx->step_grid;
    key.collide_grid = ctx->collide_grid;
    if (ctx->gexec[p][kind] && std::memcmp(&ctx->gkey[p][kind], &key, sizeof key) == 0) {
        *out = ctx->gexec[p][kind];
        return ECRIS_OK;
    }
    if (ctx->gexec[p][kind]) {
        cudaGraphExecDestroy(ctx->gexec[p][kind]);
        ctx->gexec[p][kind] = nullptr;
    }
    const bool coulomb = (ctx->h.mcc.flags & kFCoulomb) != 0;
    const uint32_t nc = (uint32_t)((size_t)ctx->h.nx * ctx->h.ny * ctx->h.nz);
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    // kind 0, the whole step; kind 1, the collision kernels alone (timed
    // steps launch the step kernel on its own before them).  With collisions
    // the scan kernel also runs the leaver pass.
    if (kind == 0) {
        e = launch_step(*ctx->h_run, ctx->ntiles, ctx->step_grid, ctx->stream);
        if (e == cudaSuccess && !coulomb) e = launch_leave(*ctx->h_run, ctx->d_ticket, 1, ctx->stream);
    }
    if (e == cudaSuccess && coulomb)
        e = launch_coulomb(*ctx->h_run, nc, ctx->ntiles, ctx->d_ticket, ctx->collide_grid, (uint32_t)kLeaveBlocks,
                           1, ctx->stream);
    const cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
    CK(e);
    CK(e2);
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    ctx->gexec[p][kind] = x;
    ctx->gkey[p][kind] = key;
    *out = x;
    return ECRIS_OK;
}

// Regroup the particles by (ion/atom, cell) into the other set of arrays and
// make that set current.  Needs the parameter block of the current set.
ecris_status sort_particles(ecris_ctx* ctx)
{
    ParticleSet dst;
    dst.x = reinterpret_cast<int32_t*>(ctx->d_soa2[0]);
    dst.y = reinterpret_cast<int32_t*>(ctx->d_soa2[1]);
    dst.z = reinterpret_cast<int32_t*>(ctx->d_soa2[2]);
    dst.vx = ctx->d_soa2[3];
    dst.vy = ctx->d_soa2[4];
    dst.vz = ctx->d_soa2[5];
    dst.meta = ctx->d_meta2;
    dst.id = ctx->d_id2;
    // the first sort after a load sees the load order: it moves 32-byte
    // records through a scratch buffer taken from the stream's pool for it
    const size_t cap4 = 4 * ctx->n4;
    uint4* aos = nullptr;
    if (ctx->fresh) CK(cudaMallocAsync((void**)&aos, 2 * cap4 * sizeof(uint4), ctx->stream));
    CK(timed(ctx, kKindOther, [&] {
        return launch_sort(*ctx->h_run, (uint32_t)cap4, dst, ctx->d_hist, ctx->d_hoff, ctx->d_hblk, aos,
                           ctx->stream);
    }, aos ? 7 : 6));
    if (aos) CK(cudaFreeAsync(aos, ctx->stream));
    for (int k = 0; k < 6; ++k) std::swap(ctx->d_soa[k], ctx->d_soa2[k]);
    std::swap(ctx->d_meta, ctx->d_meta2);
    std::swap(ctx->d_id, ctx->d_id2);
    RunDev& R = *ctx->h_run;
    R.x = reinterpret_cast<int32_t*>(ctx->d_soa[0]);
    R.y = reinterpret_cast<int32_t*>(ctx->d_soa[1]);
    R.z = reinterpret_cast<int32_t*>(ctx->d_soa[2]);
    R.vx = ctx->d_soa[3];
    R.vy = ctx->d_soa[4];
    R.vz = ctx->d_soa[5];
    R.meta = ctx->d_meta;
    R.id = ctx->d_id;
    ctx->since_sort = 0;
    ctx->fresh = false;
    ctx->parity ^= 1;
    return ECRIS_OK;
}

}  // namespace

extern "C" {

ecris_status ecris_create(ecris_ctx** out, int device, void* cuda_stream)
{
    if (!out) {
        g_create_error = "ecris_create: out is NULL";
        return ECRIS_EINVAL;
    }
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) {
        g_create_error = std::string("ecris_create: no CUDA device ") + std::to_string(device) +
                         (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : std::string());
        return e != cudaSuccess ? ECRIS_ECUDA : ECRIS_EINVAL;
    }
    ecris_ctx* ctx = new (std::nothrow) ecris_ctx();
    if (!ctx) {
        g_create_error = "ecris_create: out of host memory";
        return ECRIS_ENOMEM;
    }
    ctx->device = device;
    e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) {
        if (cuda_stream) {
            ctx->stream = (cudaStream_t)cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
            ctx->own_stream = (e == cudaSuccess);
        }
    }
    if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->h_run, sizeof(RunDev));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->h_kdt, kGateWord * sizeof(float));
    if (e != cudaSuccess) {
        g_create_error = std::string("ecris_create: ") + cudaGetErrorString(e);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        if (ctx->h_run) cudaFreeHost(ctx->h_run);
        delete ctx;
        return ECRIS_ECUDA;
    }
    ctx->step_grid = ctx->sm_count * step_blocks_per_sm();   // one wave of resident blocks
    ctx->collide_grid = ctx->sm_count * collide_blocks_per_sm();
    *out = ctx;
    return ECRIS_OK;
}

void ecris_destroy(ecris_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    free_ions(ctx);
    free_fields(ctx);
    cudaStreamSynchronize(ctx->stream);
    ctx->timer.release();
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    if (ctx->h_run) cudaFreeHost(ctx->h_run);
    if (ctx->h_kdt) cudaFreeHost(ctx->h_kdt);
    delete ctx;
}

const char* ecris_last_error(const ecris_ctx* ctx)
{
    if (!ctx) return g_create_error.c_str();
    return ctx->err.c_str();
}

ecris_status ecris_init_fields(ecris_ctx* ctx, const ecris_geometry* geo, const ecris_bfield* bf,
                               const ecris_grid* grid, const ecris_species* sp, const ecris_mcc* mcc)
{
    if (!ctx) return ECRIS_EINVAL;
    if (!geo || !bf || !grid || !sp || !mcc) return fail(ctx, ECRIS_EINVAL, "init_fields: NULL argument");
    if (!finite_pos(geo->R0) || !finite_pos(geo->L) || !finite_pos(geo->r_ap) || !(geo->r_ap < geo->R0))
        return fail(ctx, ECRIS_EINVAL, "init_fields: need R0 > r_ap > 0 and L > 0");
    {
        const double ix = geo->inlet[0], iy = geo->inlet[1], iz = geo->inlet[2];
        if (!(ix * ix + iy * iy < geo->R0 * geo->R0) || !(iz > 0.0) || !(iz < geo->L))
            return fail(ctx, ECRIS_EINVAL, "init_fields: gas inlet must lie inside the chamber");
    }
    if (bf->n_axial != 0) {
        if (bf->n_axial < 4 || bf->n_axial > 65537 || !bf->B_axial)
            return fail(ctx, ECRIS_EINVAL, "init_fields: the axial table needs 4 <= n_axial <= 65537 samples");
        for (int32_t k = 0; k < bf->n_axial; ++k)
            if (!(std::isfinite(bf->B_axial[k]) && bf->B_axial[k] >= 0.0))
                return fail(ctx, ECRIS_EINVAL, "init_fields: axial sample %d must be finite and >= 0", (int)k);
    } else if (!(std::isfinite(bf->B_min) && bf->B_min >= 0.0) || !(bf->B_inj > bf->B_min) ||
               !(bf->B_ext > bf->B_min) || !std::isfinite(bf->B_inj) || !std::isfinite(bf->B_ext)) {
        return fail(ctx, ECRIS_EINVAL, "init_fields: need B_inj > B_min >= 0 and B_ext > B_min");
    }
    if (!std::isfinite(bf->B_hex) || !std::isfinite(bf->B_ecr))
        return fail(ctx, ECRIS_EINVAL, "init_fields: B_hex and B_ecr must be finite");
    if (grid->nx < 2 || grid->ny < 2 || grid->nz < 2 ||
        (double)grid->nx * grid->ny * grid->nz > 4.0e8)
        return fail(ctx, ECRIS_EINVAL, "init_fields: mesh sizes must be >= 2 and Nc <= 4e8");
    if (!(grid->ne_in_cm3 >= 0.0) || !(grid->ne_out_cm3 >= 0.0) || !std::isfinite(grid->ne_in_cm3) ||
        !std::isfinite(grid->ne_out_cm3) || !finite_pos(grid->Te_warm_eV) || !finite_pos(grid->Te_cold_eV))
        return fail(ctx, ECRIS_EINVAL, "init_fields: need n_e >= 0 and T_e > 0");
    if ((mcc->flags & kFCoulomb) && (double)grid->nx * grid->ny * grid->nz >= 67108864.0)
        return fail(ctx, ECRIS_EINVAL, "init_fields: Coulomb collisions need Nc < 2^26 cells");
    if (!finite_pos(sp->mass_amu) || sp->qmax < 1 || sp->qmax > 63 || !sp->ip_eV || !sp->n_outer)
        return fail(ctx, ECRIS_EINVAL, "init_fields: need mass > 0, 1 <= qmax <= 63, ip and n_outer");
    for (int q = 0; q < sp->qmax; ++q)
        if (!finite_pos(sp->ip_eV[q]) || sp->n_outer[q] < 1)
            return fail(ctx, ECRIS_EINVAL, "init_fields: ionisation potential %d must be > 0 with q >= 1", q);
    if (!(mcc->n0_cm3 >= 0.0) || !std::isfinite(mcc->n0_cm3) || !finite_pos(mcc->T0_eV) ||
        !(mcc->sigma1_cm2 >= 0.0) || !(mcc->E_cx_eV >= 0.0) || !(mcc->lnL_ii >= 0.0) ||
        !(mcc->lnL_ei >= 0.0) || (mcc->ei_charge_power != 1 && mcc->ei_charge_power != 2) ||
        (mcc->flags & ~kFlagMask) || !(mcc->T_refl_eV >= 0.0) || !std::isfinite(mcc->T_refl_eV) ||
        !(mcc->sigma_el1_cm2 >= 0.0) || !std::isfinite(mcc->sigma_el1_cm2) || !(mcc->k2_factor >= 0.0) ||
        !std::isfinite(mcc->k2_factor) || !(mcc->k3_factor >= 0.0) || !std::isfinite(mcc->k3_factor))
        return fail(ctx, ECRIS_EINVAL, "init_fields: invalid collision parameters");

    CK(cudaSetDevice(ctx->device));
    free_ions(ctx);
    free_fields(ctx);
    HostRun& h = ctx->h;
    h.has_e = false;
    h.geo = *geo;
    h.bf = *bf;
    h.nx = grid->nx;
    h.ny = grid->ny;
    h.nz = grid->nz;
    h.ne_in = grid->ne_in_cm3;
    h.ne_out = grid->ne_out_cm3;
    h.Te_w = grid->Te_warm_eV;
    h.Te_c = grid->Te_cold_eV;
    h.mass_amu = sp->mass_amu;
    h.qmax = sp->qmax;
    h.ip.assign(sp->ip_eV, sp->ip_eV + sp->qmax);
    h.nout.assign(sp->n_outer, sp->n_outer + sp->qmax);
    h.mcc = *mcc;
    h.ax_y.clear();
    h.ax_M.clear();
    if (bf->n_axial) {
        h.ax_y.assign(bf->B_axial, bf->B_axial + bf->n_axial);
        axial_spline(h.ax_y, geo->L, h.ax_M);
        h.bf.n_axial = 0;          // the copy above owns the samples
        h.bf.B_axial = nullptr;
        h.zm = 0.5 * geo->L;       // (mirror constants unused with a table)
    } else {
        h.zm = geo->L / (1.0 + std::sqrt((bf->B_ext - bf->B_min) / (bf->B_inj - bf->B_min)));
    }
    for (int zone = 0; zone < 2; ++zone) {
        h.rate[zone].resize(sp->qmax);
        const double Te = zone ? h.Te_w : h.Te_c;
        for (int q = 0; q < sp->qmax; ++q) h.rate[zone][q] = lotz_rate(h.ip[q], h.nout[q], Te);
        // double ionisation (the fit of [22] is not available): k2_factor
        // times the Lotz-Maxwellian rate with threshold P_Q + P_{Q+1}
        h.rate2[zone].assign(sp->qmax, 0.0);
        if (mcc->flags & kFDouble)
            for (int q = 0; q + 1 < sp->qmax; ++q)
                h.rate2[zone][q] = mcc->k2_factor * lotz_rate(h.ip[q] + h.ip[q + 1], h.nout[q], Te);
        // triple ionisation (the scaling of [23] is not available): k3_factor
        // times the same with threshold P_Q + P_{Q+1} + P_{Q+2}
        h.rate3[zone].assign(sp->qmax, 0.0);
        if ((mcc->flags & kFDouble) && mcc->k3_factor > 0.0)
            for (int q = 0; q + 2 < sp->qmax; ++q)
                h.rate3[zone][q] =
                    mcc->k3_factor * lotz_rate(h.ip[q] + h.ip[q + 1] + h.ip[q + 2], h.nout[q], Te);
        // radiative recombination (the datasets [21] are not available):
        // Seaton's hydrogenic rate for charge Z = Q, lambda = 157890 Z^2 / T(K)
        h.rate_r[zone].assign(sp->qmax + 1, 0.0);
        for (int q = 1; q <= sp->qmax; ++q) {
            const double lam = 157890.0 * q * q / (Te * 11604.518);
            h.rate_r[zone][q] = 5.197e-14 * q * std::sqrt(lam) *
                                (0.4288 + 0.5 * std::log(lam) + 0.469 * std::pow(lam, -1.0 / 3.0)) * 1e-6;
        }
    }

    // per-cell electron data in FP64: zone by |B| at the centre, n_e, delta
    const size_t nc = (size_t)h.nx * h.ny * h.nz;
    const double dx = 2.0 * geo->R0 / h.nx, dy = 2.0 * geo->R0 / h.ny, dz = geo->L / h.nz;
    std::vector<double> ne(nc), bm(nc);
    std::vector<unsigned char> zone(nc);
    for (int iz = 0; iz < h.nz; ++iz)
        for (int iy = 0; iy < h.ny; ++iy)
            for (int ix = 0; ix < h.nx; ++ix) {
                const size_t c = ((size_t)iz * h.ny + iy) * h.nx + ix;
                const double b = bmag_host(h, -geo->R0 + (ix + 0.5) * dx, -geo->R0 + (iy + 0.5) * dy,
                                           (iz + 0.5) * dz);
                bm[c] = b;
                zone[c] = b < bf->B_ecr;
                const double nin = grid->ne_in_cells ? (double)grid->ne_in_cells[c] : grid->ne_in_cm3;
                if (zone[c] && !(nin >= 0.0 && std::isfinite(nin)))
                    return fail(ctx, ECRIS_EINVAL, "init_fields: ne_in_cells[%zu] must be finite and >= 0", c);
                ne[c] = 1e6 * (zone[c] ? nin : grid->ne_out_cm3);
            }
    h.bmag = bm;
    std::vector<float4> cell;
    cell_records(h, ne, zone, cell);
    std::vector<float4> E(nc, make_float4(0.f, 0.f, 0.f, 0.f));
    if (grid->E) {
        for (size_t c = 0; c < nc; ++c) {
            const float ex = grid->E[3 * c], ey = grid->E[3 * c + 1], ez = grid->E[3 * c + 2];
            if (!std::isfinite(ex) || !std::isfinite(ey) || !std::isfinite(ez))
                return fail(ctx, ECRIS_EINVAL, "init_fields: E[%zu] is not finite", c);
            E[c] = make_float4(ex, ey, ez, 0.f);
            if (ex != 0.0f || ey != 0.0f || ez != 0.0f) h.has_e = true;
        }
    }
    CK(cudaMallocAsync((void**)&ctx->d_cell, nc * sizeof(float4), ctx->stream));
    CK(cudaMallocAsync((void**)&ctx->d_E, nc * sizeof(float4), ctx->stream));
    CK(cudaMallocAsync((void**)&ctx->d_kdt, kKdtWords * sizeof(float), ctx->stream));
    CK(cudaMallocAsync((void**)&ctx->d_rlc, nc * sizeof(double), ctx->stream));
    // R_L n_e per cell for the device's rebuild of delta, in the order the
    // host's records take it: 2.38e-6 sqrt(T_e) / (B dX)
    std::vector<double> rlc(nc);
    for (size_t c = 0; c < nc; ++c)
        rlc[c] = 2.38e-6 * std::sqrt(zone[c] ? h.Te_w : h.Te_c) / (h.bmag[c] * dx);
    // the gate word (set with the first rate table) and the largest n_e of each zone
    const uint32_t gate_words[4] = {0xFFFFFFFFu, float_bits(h.ne_max[0]), float_bits(h.ne_max[1]), 0u};
    // the table's cubics in t per segment, from the FP64 spline:
    // a = y_k, b = y_{k+1} - y_k - h^2 (2 M_k + M_{k+1})/6, c = h^2 M_k/2,
    // d = h^2 (M_{k+1} - M_k)/6
    std::vector<float4> btab;
    if (!h.ax_y.empty()) {
        const size_t nseg = h.ax_y.size() - 1;
        const double hz = geo->L / (double)nseg;
        btab.resize(nseg);
        for (size_t k = 0; k < nseg; ++k) {
            const double y0 = h.ax_y[k], y1 = h.ax_y[k + 1], m0 = h.ax_M[k], m1 = h.ax_M[k + 1];
            btab[k] = make_float4((float)y0, (float)(y1 - y0 - hz * hz * (2.0 * m0 + m1) / 6.0),
                                  (float)(hz * hz * m0 / 2.0), (float)(hz * hz * (m1 - m0) / 6.0));
        }
        CK(cudaMallocAsync((void**)&ctx->d_btab, nseg * sizeof(float4), ctx->stream));
        CK(cudaMemcpyAsync(ctx->d_btab, btab.data(), nseg * sizeof(float4), cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(cudaMallocAsync((void**)&ctx->d_nanbu, kNanbuN * sizeof(float), ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_nanbu, nanbu_table(), kNanbuN * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_cell, cell.data(), nc * sizeof(float4), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_rlc, rlc.data(), nc * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_kdt + kGateWord, gate_words, sizeof gate_words, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_E, E.data(), nc * sizeof(float4), cudaMemcpyHostToDevice, ctx->stream));
    // the host vectors die at return: wait for the copies
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->have_fields = true;
    ctx->ne_device = false;
    ctx->failed = false;
    ctx->err.clear();
    return ECRIS_OK;
}

ecris_status ecris_load_ions(ecris_ctx* ctx, size_t n, const float* const xyzv[6], const uint8_t* q,
                             double weight, uint64_t seed, int src_is_device)
{
    if (!ctx) return ECRIS_EINVAL;
    if (!ctx->have_fields) return fail(ctx, ECRIS_ESTATE, "load_ions: call ecris_init_fields first");
    if (!finite_pos(weight)) return fail(ctx, ECRIS_EINVAL, "load_ions: weight must be > 0");
    const HostRun& h = ctx->h;
    if ((double)n * (double)(h.qmax > 1 ? h.qmax : 1) >= 4294967296.0 || n > 0xFFFFFFF0ull)
        return fail(ctx, ECRIS_EINVAL, "load_ions: n * qmax must stay below 2^32 (packed deposit)");
    if (n > 0) {
        if (!xyzv || !q) return fail(ctx, ECRIS_EINVAL, "load_ions: NULL particle arrays");
        for (int k = 0; k < 6; ++k)
            if (!xyzv[k]) return fail(ctx, ECRIS_EINVAL, "load_ions: NULL particle array %d", k);
    }
    CK(cudaSetDevice(ctx->device));
    const size_t n4 = (n + 3) / 4;
    const size_t cap = n4 > 0 ? 4 * n4 : 4;
    const size_t nc = (size_t)h.nx * h.ny * h.nz;
    // device buffers are kept across loads while they are large enough
    if (!ctx->have_ions || cap > ctx->cap || nc != ctx->cap_cells) {
        free_ions(ctx);
        for (int k = 0; k < 6; ++k)
            CK(cudaMallocAsync((void**)&ctx->d_soa[k], cap * sizeof(float), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_meta, cap * sizeof(uint32_t), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_id, cap * sizeof(uint32_t), ctx->stream));
        for (int k = 0; k < 6; ++k)
            CK(cudaMallocAsync((void**)&ctx->d_soa2[k], cap * sizeof(float), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_meta2, cap * sizeof(uint32_t), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_id2, cap * sizeof(uint32_t), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_hist, (2 * nc + 1) * sizeof(uint32_t), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_hoff, (2 * nc + 2) * sizeof(uint32_t), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_hblk, (size_t)sort_scan_blocks((uint32_t)(2 * nc + 1)) * sizeof(uint32_t),
                           ctx->stream));
        CK(cudaMemsetAsync(ctx->d_hist, 0, (2 * nc + 1) * sizeof(uint32_t), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_q8, cap, ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_dep, nc * sizeof(unsigned long long), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_count, nc * sizeof(unsigned long long), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_charge, nc * sizeof(unsigned long long), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_mark, nc * sizeof(unsigned long long), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_ne64, nc * sizeof(double), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_tally, kTallyWords * sizeof(unsigned long long), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_census, kQSlots * sizeof(unsigned long long), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_step, sizeof(uint32_t), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_leave, cap * sizeof(uint32_t), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_birth, cap * sizeof(uint32_t), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_fptd, kFptdWords * sizeof(unsigned long long), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_nleave, sizeof(uint32_t), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_ticket, sizeof(unsigned int), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_bad, 2 * sizeof(unsigned int), ctx->stream));
        CK(cudaMallocAsync((void**)&ctx->d_err, sizeof(uint32_t), ctx->stream));
        if (h.mcc.flags & kFCoulomb) {
            // participant lists for tiles of up to kMaxTile particles
            const size_t slots = cap + kMaxTile;
            CK(cudaMallocAsync((void**)&ctx->d_plist, slots * sizeof(uint4), ctx->stream));
            CK(cudaMallocAsync((void**)&ctx->d_cslot, cap * sizeof(uint32_t), ctx->stream));
            CK(cudaMallocAsync((void**)&ctx->d_sslot, cap * sizeof(uint32_t), ctx->stream));
            CK(cudaMallocAsync((void**)&ctx->d_pvel, slots * sizeof(float4), ctx->stream));
            CK(cudaMallocAsync((void**)&ctx->d_tcount, (cap / kMinTile + 1) * sizeof(uint32_t), ctx->stream));
            CK(cudaMallocAsync((void**)&ctx->d_ckeys, cap * sizeof(unsigned long long), ctx->stream));
            CK(cudaMallocAsync((void**)&ctx->d_crec, cap * sizeof(float4), ctx->stream));
            CK(cudaMallocAsync((void**)&ctx->d_ccount, nc * sizeof(uint32_t), ctx->stream));
            CK(cudaMallocAsync((void**)&ctx->d_cstart, (cap / kCellIonsMin + 2) * sizeof(uint32_t), ctx->stream));
            CK(cudaMallocAsync((void**)&ctx->d_crange, 2 * sizeof(uint32_t), ctx->stream));
            CK(cudaMallocAsync((void**)&ctx->d_coff, (nc + 1) * sizeof(uint32_t), ctx->stream));
            CK(cudaMallocAsync((void**)&ctx->d_cstat, (size_t)(coulomb_scan_blocks((uint32_t)nc) + 1) * sizeof(unsigned long long),
                               ctx->stream));
        }
        ctx->cap = cap;
        ctx->cap_cells = nc;
        ctx->have_ions = true;
    }
    ctx->n = n;
    ctx->n4 = n4;
    ctx->ntiles = (uint32_t)((n4 + kTileGroups - 1) / kTileGroups);
    const cudaMemcpyKind kind = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (n) {
        for (int k = 0; k < 6; ++k)
            CK(cudaMemcpyAsync(ctx->d_soa[k], xyzv[k], n * sizeof(float), kind, ctx->stream));
        CK(cudaMemcpyAsync(ctx->d_q8, q, n, kind, ctx->stream));
    }
    if (ctx->d_ccount) CK(cudaMemsetAsync(ctx->d_ccount, 0, nc * sizeof(uint32_t), ctx->stream));
    if (ctx->d_crange) {
        static const uint32_t crange0[2] = {(uint32_t)kCellIons, 0u};
        CK(cudaMemcpyAsync(ctx->d_crange, crange0, sizeof crange0, cudaMemcpyHostToDevice, ctx->stream));
    }
    if (ctx->d_cstat)
        CK(cudaMemsetAsync(ctx->d_cstat, 0, (size_t)(coulomb_scan_blocks((uint32_t)nc) + 1) * sizeof(unsigned long long),
                           ctx->stream));
    CK(cudaMemsetAsync(ctx->d_dep, 0, nc * sizeof(unsigned long long), ctx->stream));
    CK(cudaMemsetAsync(ctx->d_count, 0, nc * sizeof(unsigned long long), ctx->stream));
    CK(cudaMemsetAsync(ctx->d_charge, 0, nc * sizeof(unsigned long long), ctx->stream));
    CK(cudaMemsetAsync(ctx->d_mark, 0, nc * sizeof(unsigned long long), ctx->stream));
    CK(cudaMemsetAsync(ctx->d_tally, 0, kTallyWords * sizeof(unsigned long long), ctx->stream));
    CK(cudaMemsetAsync(ctx->d_birth, 0xFF, ctx->cap * sizeof(uint32_t), ctx->stream));   // births unknown
    CK(cudaMemsetAsync(ctx->d_fptd, 0, kFptdWords * sizeof(unsigned long long), ctx->stream));
    {
        const ecris_status pst = zero_probes(ctx);
        if (pst != ECRIS_OK) return pst;
    }
    CK(cudaMemsetAsync(ctx->d_step, 0, sizeof(uint32_t), ctx->stream));
    CK(cudaMemsetAsync(ctx->d_nleave, 0, sizeof(uint32_t), ctx->stream));
    CK(cudaMemsetAsync(ctx->d_ticket, 0, sizeof(unsigned int), ctx->stream));
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), ctx->stream));
    CK(cudaMemsetAsync(ctx->d_bad, 0, sizeof(unsigned int), ctx->stream));
    CK(cudaMemsetAsync(ctx->d_bad + 1, 0xFF, sizeof(unsigned int), ctx->stream));
    // validate on the device, build the meta words and fill the padding slots
    LoadCheck lc;
    lc.R0sq = (float)(h.geo.R0 * h.geo.R0);
    lc.L = (float)h.geo.L;
    lc.qmax = (uint32_t)h.qmax;
    lc.inlet_x = (float)h.geo.inlet[0];
    lc.inlet_y = (float)h.geo.inlet[1];
    lc.inlet_z = (float)h.geo.inlet[2];
    {
        const double a = 2147483648.0 / h.geo.R0, b = 4294967296.0 / h.geo.L;
        lc.inv_sxy_hi = (float)a;
        lc.inv_sxy_lo = (float)(a - (double)lc.inv_sxy_hi);
        lc.inv_sz_hi = (float)b;
        lc.inv_sz_lo = (float)(b - (double)lc.inv_sz_hi);
    }
    CK(launch_load_init(lc, ctx->d_soa, ctx->d_q8, ctx->d_meta, ctx->d_id, (uint32_t)n, (uint32_t)cap, ctx->d_bad,
                        ctx->stream));
    unsigned int bad[2] = {0u, 0u};
    CK(cudaMemcpyAsync(bad, ctx->d_bad, sizeof bad, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (bad[0]) {
        ctx->n = 0;
        ctx->n4 = 0;
        ctx->ntiles = 0;
        ctx->loaded = false;
        return fail(ctx, ECRIS_EINVAL,
                    "load_ions: %u particle(s) outside the chamber, not finite or with Q > qmax "
                    "(first index %u)", bad[0], bad[1]);
    }
    ctx->weight = weight;
    ctx->seed = seed;
    ctx->steps_done = 0;
    ctx->h.steps_mark = 0;
    ctx->time_s = 0.0;
    ctx->dt_loaded = -1.0;
    ctx->since_fold = 0;
    // a load leaves the particles in load order.  The first ecris_step call
    // after it groups them first only if it runs kSortAfterLoad or more
    // steps; a shorter first call (a load, a step and a read-back, say) steps
    // them as they are, and the next call sorts (the sort costs several
    // steps' time)
    ctx->since_sort = 0;
    ctx->fresh = true;
    ctx->calls_since_load = 0;
    // fold the packed deposit before its low word (charge) can carry
    const double per_step = (double)(n ? n : 1) * (h.qmax > 1 ? h.qmax : 1);
    const double k = std::floor(4294967295.0 / per_step);
    ctx->fold_every = (uint32_t)(k < 1.0 ? 1.0 : (k > 1e6 ? 1e6 : k));
    ctx->loaded = true;
    ctx->failed = false;
    ctx->err.clear();
    return ECRIS_OK;
}

ecris_status ecris_step(ecris_ctx* ctx, uint32_t nsteps, double dt)
{
    if (!ctx) return ECRIS_EINVAL;
    if (ctx->failed) return fail(ctx, ECRIS_ESTATE, "step: context failed earlier (%s); reload", ctx->err.c_str());
    if (!ctx->loaded) return fail(ctx, ECRIS_ESTATE, "step: call ecris_load_ions first");
    if (!finite_pos(dt)) return fail(ctx, ECRIS_EINVAL, "step: dt must be finite and > 0");
    if (ctx->steps_done + nsteps >= kMaxSteps)
        return fail(ctx, ECRIS_EINVAL, "step: more than 2^30 steps since load");
    CK(cudaSetDevice(ctx->device));
    ecris_status st = upload_dt(ctx, dt);
    if (st != ECRIS_OK) return st;
    const bool coulomb = (ctx->h.mcc.flags & kFCoulomb) != 0;
    const uint32_t nc = (uint32_t)((size_t)ctx->h.nx * ctx->h.ny * ctx->h.nz);
    for (uint32_t s = 0; s < nsteps; ++s) {
        const bool due = ctx->since_sort >= ctx->sort_every ||
                         (ctx->fresh && s == 0 && (nsteps >= kSortAfterLoad || ctx->calls_since_load > 0));
        if (due && ctx->n4 > 0) {
            st = sort_particles(ctx);
            if (st != ECRIS_OK) return st;
        }
        if (!ctx->timer.on) {
            // the whole step as one graph launch
            cudaGraphExec_t x = nullptr;
            st = step_graph(ctx, 0, &x);
            if (st != ECRIS_OK) return st;
            CK(cudaGraphLaunch(x, ctx->stream));
        } else {
            // timed: the step kernel on its own, the collision kernels as a graph
            CK(timed(ctx, kKindStep, [&] {
                return launch_step(*ctx->h_run, ctx->ntiles, ctx->step_grid, ctx->stream);
            }));
            if (!coulomb)
                CK(timed(ctx, kKindOther, [&] { return launch_leave(*ctx->h_run, ctx->d_ticket, 1, ctx->stream); }));
            if (coulomb) {
                cudaGraphExec_t x = nullptr;
                st = step_graph(ctx, 1, &x);
                if (st != ECRIS_OK) return st;
                CK(timed(ctx, kKindCoulomb, [&] { return cudaGraphLaunch(x, ctx->stream); }, kCoulombKernels));
            }
        }
        if (++ctx->since_fold >= ctx->fold_every) {
            CK(timed(ctx, kKindOther, [&] {
                return launch_fold(*ctx->h_run, nc, ctx->d_count, ctx->d_charge, ctx->stream);
            }));
            ctx->since_fold = 0;
        }
        ++ctx->since_sort;
    }
    ctx->steps_done += nsteps;
    ++ctx->calls_since_load;
    ctx->time_s += dt * nsteps;
    return ECRIS_OK;
}

namespace {

// the diagnostics of a run from its tally words (and census, if any) after
// `steps` steps lasting time_s
void fill_diag(const HostRun& h, double weight, const unsigned long long* tally, const unsigned long long* census,
               uint64_t steps, double time_s, ecris_diag_out* out)
{
    const int Q1 = h.qmax + 1;
    out->qmax = h.qmax;
    out->steps = steps;
    out->time_s = time_s;
    for (int q = 0; q < Q1; ++q) {
        if (out->extracted) out->extracted[q] = (int64_t)tally[kTallyExtracted + q];
        if (out->lost) out->lost[q] = (int64_t)tally[kTallyLost + q];
        if (out->alive_by_q && census) out->alive_by_q[q] = (int64_t)census[q];
        if (out->current_A)
            out->current_A[q] = time_s > 0.0 ? q * kE * weight * (double)tally[kTallyExtracted + q] / time_s : 0.0;
    }
    out->ke_lost_eV = 1e-6 * (double)tally[kTallyKe];
    out->coulomb_collisions = (int64_t)tally[kTallyCoulomb];
    // power balance: kinetic + potential energy of the ions that left plus
    // 3/2 T_ew per electron that left with them
    double e_eV = out->ke_lost_eV, ipcum = 0.0;
    for (int q = 1; q < Q1; ++q) {
        ipcum += h.ip[q - 1];
        const double nleft = (double)tally[kTallyExtracted + q] + (double)tally[kTallyLost + q];
        e_eV += nleft * (ipcum + 1.5 * q * h.Te_w);
    }
    out->power_W = time_s > 0.0 ? weight * e_eV * kE / time_s : 0.0;
}

}  // namespace

ecris_status ecris_diag(ecris_ctx* ctx, ecris_diag_out* out)
{
    if (!ctx) return ECRIS_EINVAL;
    if (!out) return fail(ctx, ECRIS_EINVAL, "diag: out is NULL");
    if (!ctx->loaded) return fail(ctx, ECRIS_ESTATE, "diag: call ecris_load_ions first");
    if (ctx->failed) return fail(ctx, ECRIS_ESTATE, "diag: context failed earlier (%s)", ctx->err.c_str());
    CK(cudaSetDevice(ctx->device));
    const HostRun& h = ctx->h;
    const size_t nc = (size_t)h.nx * h.ny * h.nz;
    if (ctx->dt_loaded < 0.0) {
        ecris_status st = upload_dt(ctx, 1e-9);   // parameter block for the census kernel
        if (st != ECRIS_OK) return st;
    }
    CK(launch_fold(*ctx->h_run, (uint32_t)nc, ctx->d_count, ctx->d_charge, ctx->stream));
    ctx->since_fold = 0;
    CK(cudaMemsetAsync(ctx->d_census, 0, kQSlots * sizeof(unsigned long long), ctx->stream));
    CK(launch_census(*ctx->h_run, (uint32_t)ctx->n4, ctx->d_census, ctx->stream));
    unsigned long long tally[kTallyWords], census[kQSlots];
    uint32_t err = 0;
    CK(cudaMemcpyAsync(&err, ctx->d_err, sizeof err, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(tally, ctx->d_tally, sizeof tally, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(census, ctx->d_census, sizeof census, cudaMemcpyDeviceToHost, ctx->stream));
    if (out->cell_count)
        CK(cudaMemcpyAsync(out->cell_count, ctx->d_count, nc * 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (out->cell_charge)
        CK(cudaMemcpyAsync(out->cell_charge, ctx->d_charge, nc * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (err) {
        ctx->failed = true;
        return fail(ctx, ECRIS_ETIMEOUT, "diag: a kernel's bounded wait for its tile copies ran out; reload");
    }
    fill_diag(h, ctx->weight, tally, census, ctx->steps_done, ctx->time_s, out);
    return ECRIS_OK;
}

ecris_status ecris_update_ne(ecris_ctx* ctx)
{
    if (!ctx) return ECRIS_EINVAL;
    if (!ctx->loaded) return fail(ctx, ECRIS_ESTATE, "update_ne: call ecris_load_ions first");
    if (ctx->failed) return fail(ctx, ECRIS_ESTATE, "update_ne: context failed earlier (%s)", ctx->err.c_str());
    CK(cudaSetDevice(ctx->device));
    return update_ne(ctx);
}

ecris_status ecris_get_fptd(ecris_ctx* ctx, uint64_t* hist, uint64_t* age_sum)
{
    if (!ctx) return ECRIS_EINVAL;
    if (!ctx->loaded) return fail(ctx, ECRIS_ESTATE, "get_fptd: call ecris_load_ions first");
    CK(cudaSetDevice(ctx->device));
    return get_fptd(ctx, hist, age_sum);
}

ecris_status ecris_get_extraction_radius(ecris_ctx* ctx, double* r_sum)
{
    if (!ctx) return ECRIS_EINVAL;
    if (!r_sum) return fail(ctx, ECRIS_EINVAL, "get_extraction_radius: r_sum is NULL");
    if (!ctx->loaded) return fail(ctx, ECRIS_ESTATE, "get_extraction_radius: call ecris_load_ions first");
    CK(cudaSetDevice(ctx->device));
    return get_extraction_radius(ctx, r_sum);
}

ecris_status ecris_set_probes(ecris_ctx* ctx, const ecris_probe_spec* spec)
{
    if (!ctx) return ECRIS_EINVAL;
    if (!spec) return fail(ctx, ECRIS_EINVAL, "set_probes: spec is NULL");
    if (!ctx->have_fields) return fail(ctx, ECRIS_ESTATE, "set_probes: call ecris_init_fields first");
    return set_probes(ctx, spec);
}

ecris_status ecris_probe_sample(ecris_ctx* ctx)
{
    if (!ctx) return ECRIS_EINVAL;
    if (!ctx->loaded) return fail(ctx, ECRIS_ESTATE, "probe_sample: call ecris_load_ions first");
    if (ctx->failed) return fail(ctx, ECRIS_ESTATE, "probe_sample: context failed earlier (%s)", ctx->err.c_str());
    CK(cudaSetDevice(ctx->device));
    return probe_sample(ctx);
}

ecris_status ecris_get_probes(ecris_ctx* ctx, uint64_t* samples, double* moments, uint64_t* screens)
{
    if (!ctx) return ECRIS_EINVAL;
    CK(cudaSetDevice(ctx->device));
    return get_probes(ctx, samples, moments, screens);
}

ecris_status ecris_get_cells(ecris_ctx* ctx, float* ne, float* delta_x, float* delta_y)
{
    if (!ctx) return ECRIS_EINVAL;
    if (!ctx->have_fields) return fail(ctx, ECRIS_ESTATE, "get_cells: call ecris_init_fields first");
    CK(cudaSetDevice(ctx->device));
    return get_cells(ctx, ne, delta_x, delta_y);
}

ecris_status ecris_get_state(ecris_ctx* ctx, float* const xyzv[6], uint32_t* meta, int dst_is_device)
{
    if (!ctx) return ECRIS_EINVAL;
    if (!ctx->loaded) return fail(ctx, ECRIS_ESTATE, "get_state: call ecris_load_ions first");
    CK(cudaSetDevice(ctx->device));
    if (ctx->dt_loaded < 0.0) {
        ecris_status st = upload_dt(ctx, 1e-9);   // parameter block for the export kernel
        if (st != ECRIS_OK) return st;
    }
    const double sxy = ctx->h.geo.R0 / 2147483648.0, sz = ctx->h.geo.L / 4294967296.0;
    const size_t n = ctx->n;
    if (n) {
        // the particles sit in sorted order: scatter them back to load order
        // by their ids (into the caller's device arrays, or via the spare set)
        if (dst_is_device) {
            CK(launch_export_ordered(*ctx->h_run, (uint32_t)n, (uint32_t)(4 * ctx->n4), xyzv, meta, sxy, sz,
                                     ctx->stream));
        } else {
            float* spare[6];
            for (int k = 0; k < 6; ++k) spare[k] = (xyzv && xyzv[k]) ? ctx->d_soa2[k] : nullptr;
            CK(launch_export_ordered(*ctx->h_run, (uint32_t)n, (uint32_t)(4 * ctx->n4), spare,
                                     meta ? ctx->d_meta2 : nullptr, sxy, sz, ctx->stream));
            for (int k = 0; k < 6; ++k)
                if (spare[k])
                    CK(cudaMemcpyAsync(xyzv[k], spare[k], n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
            if (meta)
                CK(cudaMemcpyAsync(meta, ctx->d_meta2, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
        }
    }
    if (!dst_is_device) CK(cudaStreamSynchronize(ctx->stream));
    return ECRIS_OK;
}

ecris_status ecris_set_tuning(ecris_ctx* ctx, const ecris_tuning* t)
{
    if (!ctx) return ECRIS_EINVAL;
    if (!t) return fail(ctx, ECRIS_EINVAL, "set_tuning: NULL argument");
    if (t->sort_every < 1) return fail(ctx, ECRIS_EINVAL, "set_tuning: sort_every must be >= 1");
    ctx->sort_every = (uint32_t)t->sort_every;
    if (ctx->since_sort > ctx->sort_every) ctx->since_sort = ctx->sort_every;
    return ECRIS_OK;
}

ecris_status ecris_set_profiling(ecris_ctx* ctx, int enable)
{
    if (!ctx) return ECRIS_EINVAL;
    CK(cudaSetDevice(ctx->device));
    CK(ctx->timer.collect(ctx->stream));
    ctx->timer.reset(enable != 0);
    return ECRIS_OK;
}

ecris_status ecris_get_profile(ecris_ctx* ctx, ecris_profile* out)
{
    if (!ctx) return ECRIS_EINVAL;
    if (!out) return fail(ctx, ECRIS_EINVAL, "get_profile: out is NULL");
    CK(cudaSetDevice(ctx->device));
    CK(ctx->timer.collect(ctx->stream));
    ctx->timer.fill(out);
    return ECRIS_OK;
}

}  // extern "C"

// ============================================================================
// Batched form
// ============================================================================
constexpr int kBatchSideStreams = 8;

struct ecris_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sm_count = 0;
    int blocks_per_sm = 0;          // 0: as many as fit
    int shape = kDefaultShape;      // launch shape of the batched step kernel
    int max_bps[kStepShapes] = {};  // resident blocks per SM of each shape
    uint32_t sort_every = 32;
    size_t budget = 0, used = 0;
    std::string err;
    std::vector<ecris_ctx*> runs;   // by handle; nullptr: free slot
    std::vector<size_t> bytes;      // device bytes charged per run
    std::vector<double> dt;         // time step per run
    RunDev* d_runs = nullptr;       // parameter blocks by handle
    RunDev* h_runs = nullptr;       // pinned staging of the same
    cudaEvent_t staged = nullptr;   // the last upload from h_runs has finished
    size_t runs_cap = 0;
    uint2* d_items = nullptr;       // work list (handle, tile)
    size_t items_cap = 0;
    uint32_t nitems = 0;
    bool variants = false;          // some run has an opt-in process of kFVariants
    bool layout_dirty = true;       // work list must be rebuilt
    bool params_dirty = true;       // parameter blocks must be uploaded
    cudaGraphExec_t gexec = nullptr;
    bool graph_dirty = true;
    unsigned int* d_ticket = nullptr;   // last-block ticket of the leaver pass
    KernelTimer timer;              // ecris_batch_set_profiling
    // side streams on which the captured graph runs the collision kernels of
    // different runs side by side (small runs do not fill the GPU alone)
    cudaStream_t side[kBatchSideStreams] = {};
    cudaEvent_t side_join[kBatchSideStreams] = {};
    cudaEvent_t side_fork = nullptr;
    // the layout sorts of the runs due for one, spread over the same side
    // streams outside the graph, with their own fork and join events
    cudaEvent_t sort_join[kBatchSideStreams] = {};
    cudaEvent_t sort_fork = nullptr;
    // added runs are set up on their own stream, so the batch's queued steps
    // keep running meanwhile
    cudaStream_t setup = nullptr;
    // pinned staging of the work list, and the event after its last upload
    uint2* h_items = nullptr;
    size_t h_items_cap = 0;
    cudaEvent_t items_staged = nullptr;
    // graphs replaced while launches of them may still be queued, each with an
    // event recorded after its last launch; destroyed once that has passed
    std::vector<std::pair<cudaEvent_t, cudaGraphExec_t>> old_graphs;
    // pinned host blocks of removed runs (freed with the batch: freeing pinned
    // memory may synchronise the device)
    std::vector<void*> old_host;
};

namespace {

ecris_status bfail(ecris_batch* b, ecris_status st, const std::string& msg)
{
    b->err = msg;
    return st;
}

#define BCK(call)                                                                      \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? ECRIS_ENOMEM : ECRIS_ECUDA, \
                         std::string(#call) + ": " + cudaGetErrorString(e_));           \
    } while (0)

bool run_live(const ecris_batch* b, int32_t r)
{
    return r >= 0 && (size_t)r < b->runs.size() && b->runs[r] != nullptr;
}

// upload the parameter blocks of all runs (free slots get a block whose step
// pointer is NULL, which the kernels skip)
// destroy the replaced graphs whose last launch has passed
void batch_reap(ecris_batch* b)
{
    size_t k = 0;
    for (auto& g : b->old_graphs) {
        if (cudaEventQuery(g.first) == cudaSuccess) {
            cudaGraphExecDestroy(g.second);
            cudaEventDestroy(g.first);
        } else {
            b->old_graphs[k++] = g;
        }
    }
    b->old_graphs.resize(k);
}

// Release a removed run without waiting for the batch's queued steps: its
// device memory is freed in stream order after them (no launch enqueued later
// reads it), its pinned blocks are kept until the batch goes.
void batch_release_run(ecris_batch* b, ecris_ctx* c)
{
    c->stream = b->stream;
    free_ions(c);
    free_fields(c);
    c->timer.release();
    if (c->h_run) b->old_host.push_back(c->h_run);
    if (c->h_kdt) b->old_host.push_back(c->h_kdt);
    delete c;
}

ecris_status batch_upload(ecris_batch* b)
{
    const size_t nr = b->runs.size();
    if (nr > b->runs_cap) {
        // queued launches may still read the old blocks: free them in stream order
        BCK(cudaEventSynchronize(b->staged));   // the last upload has read the old staging copy
        if (b->d_runs) cudaFreeAsync(b->d_runs, b->stream);
        if (b->h_runs) b->old_host.push_back(b->h_runs);
        b->runs_cap = nr + 16;
        BCK(cudaMallocAsync((void**)&b->d_runs, b->runs_cap * sizeof(RunDev), b->stream));
        BCK(cudaMallocHost((void**)&b->h_runs, b->runs_cap * sizeof(RunDev)));
        b->graph_dirty = true;
    } else {
        BCK(cudaEventSynchronize(b->staged));   // the previous upload has read the staging copy
    }
    for (size_t r = 0; r < nr; ++r) {
        if (b->runs[r]) b->h_runs[r] = *b->runs[r]->h_run;
        else std::memset(&b->h_runs[r], 0, sizeof(RunDev));
    }
    if (nr) BCK(cudaMemcpyAsync(b->d_runs, b->h_runs, nr * sizeof(RunDev), cudaMemcpyHostToDevice, b->stream));
    BCK(cudaEventRecord(b->staged, b->stream));
    b->params_dirty = false;
    return ECRIS_OK;
}

ecris_status batch_items(ecris_batch* b)
{
    std::vector<uint2> items;
    const uint32_t tile = shape_tile(b->shape), groups = tile / 4;
    for (size_t r = 0; r < b->runs.size(); ++r) {
        ecris_ctx* c = b->runs[r];
        if (!c) continue;
        // the run's tiles in the batch's launch shape
        c->tile = tile;
        if (c->h_run->tile != tile) {
            c->h_run->tile = tile;
            b->params_dirty = true;
        }
        c->btiles = (uint32_t)((c->n4 + groups - 1) / groups);
        for (uint32_t t = 0; t < c->btiles; ++t) items.push_back(make_uint2((uint32_t)r, t));
    }
    // the last upload must have read the staging copy before it is rewritten;
    // queued launches may still read the old device list, freed in stream order
    if (b->items_staged) BCK(cudaEventSynchronize(b->items_staged));
    if (items.size() > b->items_cap) {
        if (b->d_items) cudaFreeAsync(b->d_items, b->stream);
        b->items_cap = items.size() + 1024;
        BCK(cudaMallocAsync((void**)&b->d_items, b->items_cap * sizeof(uint2), b->stream));
    }
    if (items.size() > b->h_items_cap) {
        if (b->h_items) b->old_host.push_back(b->h_items);
        b->h_items_cap = items.size() + 1024;
        BCK(cudaMallocHost((void**)&b->h_items, b->h_items_cap * sizeof(uint2)));
    }
    if (!items.empty()) {
        std::memcpy(b->h_items, items.data(), items.size() * sizeof(uint2));
        BCK(cudaMemcpyAsync(b->d_items, b->h_items, items.size() * sizeof(uint2), cudaMemcpyHostToDevice,
                            b->stream));
        BCK(cudaEventRecord(b->items_staged, b->stream));
    }
    b->nitems = (uint32_t)items.size();
    b->variants = false;
    for (auto* c : b->runs)
        if (c && ((c->h.mcc.flags & kFVariants) || !c->h.ax_y.empty())) b->variants = true;
    b->layout_dirty = false;
    b->graph_dirty = true;
    return ECRIS_OK;
}

// one step of every run: the batched step kernel, the collision kernels of
// the runs that have them, and the step counters of the others
int batch_bps(const ecris_batch* b)
{
    const int m = b->max_bps[b->shape];
    return b->blocks_per_sm > 0 ? std::min(b->blocks_per_sm, m) : m;
}

cudaError_t batch_side_streams(ecris_batch* b)
{
    if (b->side_fork) return cudaSuccess;
    cudaError_t e = cudaEventCreateWithFlags(&b->side_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->sort_fork, cudaEventDisableTiming);
    for (int k = 0; e == cudaSuccess && k < kBatchSideStreams; ++k) {
        e = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->side_join[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->sort_join[k], cudaEventDisableTiming);
    }
    return e;
}

// The step of every run (captured into the batch graph): the batched step
// kernel and leaver pass on the batch stream (the leaver pass advances the
// step counters of the runs without collisions between ions); the collision
// kernels of the runs that have them forked onto the side streams, so
// different runs' collision kernels overlap, and joined back.
cudaError_t batch_launch(ecris_batch* b)
{
    cudaError_t e = launch_step_batch(b->d_runs, b->d_items, b->nitems, b->sm_count * batch_bps(b), b->variants,
                                      b->shape, b->stream);
    if (e == cudaSuccess) e = launch_leave_batch(b->d_runs, (uint32_t)b->runs.size(), b->d_ticket, b->stream);
    if (e == cudaSuccess) e = batch_side_streams(b);
    if (e == cudaSuccess) e = cudaEventRecord(b->side_fork, b->stream);
    int used = 0;
    for (size_t r = 0; e == cudaSuccess && r < b->runs.size(); ++r) {
        ecris_ctx* c = b->runs[r];
        if (!c || !(c->h.mcc.flags & kFCoulomb)) continue;
        const int k = used % kBatchSideStreams;
        if (used < kBatchSideStreams) e = cudaStreamWaitEvent(b->side[k], b->side_fork, 0);
        ++used;
        const uint32_t nc = (uint32_t)((size_t)c->h.nx * c->h.ny * c->h.nz);
        if (e == cudaSuccess)
            e = launch_coulomb(*c->h_run, nc, c->btiles, c->d_ticket, c->collide_grid, 0u, 0, b->side[k]);
    }
    for (int k = 0; e == cudaSuccess && k < used && k < kBatchSideStreams; ++k) {
        e = cudaEventRecord(b->side_join[k], b->side[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->side_join[k], 0);
    }
    return e;
}

ecris_status batch_graph(ecris_batch* b)
{
    if (!b->graph_dirty && b->gexec) return ECRIS_OK;
    if (b->gexec) {
        // launches of the old graph may still be queued: destroy it later
        cudaEvent_t ev = nullptr;
        BCK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        BCK(cudaEventRecord(ev, b->stream));
        b->old_graphs.emplace_back(ev, b->gexec);
        b->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    const cudaError_t e = batch_launch(b);
    const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    BCK(e);
    BCK(e2);
    const cudaError_t e3 = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    BCK(e3);
    b->graph_dirty = false;
    return ECRIS_OK;
}

}  // namespace

extern "C" {

size_t ecris_run_bytes(size_t n, int32_t nx, int32_t ny, int32_t nz, int coulomb)
{
    const size_t cap = 4 * ((n + 3) / 4) + 4;
    const size_t nc = (size_t)(nx > 0 ? nx : 0) * (ny > 0 ? ny : 0) * (nz > 0 ? nz : 0);
    // two particle sets with ids, the first sort's records (held while it
    // runs), leaver list, births, load bytes, Coulomb lists
    size_t per_p = 2 * 32 + 32 + 4 + 4 + 4 + 1;
    if (coulomb) per_p += 16 + 16 + 8 + 16 + 4 + 4 + 1;
    // cell records, E, deposit, time sums, sort histogram and scan, the n_e
    // update's mark, scratch and R_L coefficients, Coulomb counts
    size_t per_c = 16 + 16 + 8 + 8 + 8 + 4 + 4 + 8 + 8 + 8 + (coulomb ? 12 : 0);
    return cap * per_p + nc * per_c + (1u << 20);
}

ecris_status ecris_batch_create(ecris_batch** out, int device, void* cuda_stream, size_t hbm_budget_bytes)
{
    if (!out) {
        g_create_error = "batch_create: out is NULL";
        return ECRIS_EINVAL;
    }
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        g_create_error = "batch_create: no such CUDA device";
        return ECRIS_EINVAL;
    }
    ecris_batch* b = new (std::nothrow) ecris_batch();
    if (!b) return ECRIS_ENOMEM;
    b->device = device;
    b->budget = hbm_budget_bytes;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) {
        if (cuda_stream) {
            b->stream = (cudaStream_t)cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
            b->own_stream = e == cudaSuccess;
        }
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->items_staged, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->setup, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&b->d_ticket, sizeof(unsigned int), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ticket, 0, sizeof(unsigned int), b->stream);
    if (e != cudaSuccess) {
        g_create_error = std::string("batch_create: ") + cudaGetErrorString(e);
        if (b->d_ticket) cudaFreeAsync(b->d_ticket, b->stream);
        if (b->staged) cudaEventDestroy(b->staged);
        if (b->items_staged) cudaEventDestroy(b->items_staged);
        if (b->setup) cudaStreamDestroy(b->setup);
        if (b->own_stream) cudaStreamDestroy(b->stream);
        delete b;
        return ECRIS_ECUDA;
    }
    for (int k = 0; k < kStepShapes; ++k) b->max_bps[k] = step_batch_blocks_per_sm(k);
    *out = b;
    return ECRIS_OK;
}

void ecris_batch_destroy(ecris_batch* b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    for (auto* c : b->runs)
        if (c) ecris_destroy(c);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->d_runs) cudaFreeAsync(b->d_runs, b->stream);
    if (b->d_items) cudaFreeAsync(b->d_items, b->stream);
    if (b->d_ticket) cudaFreeAsync(b->d_ticket, b->stream);
    cudaStreamSynchronize(b->stream);
    for (int k = 0; k < kBatchSideStreams; ++k) {
        if (b->side[k]) cudaStreamDestroy(b->side[k]);
        if (b->side_join[k]) cudaEventDestroy(b->side_join[k]);
        if (b->sort_join[k]) cudaEventDestroy(b->sort_join[k]);
    }
    if (b->side_fork) cudaEventDestroy(b->side_fork);
    if (b->sort_fork) cudaEventDestroy(b->sort_fork);
    for (auto& g : b->old_graphs) {
        cudaGraphExecDestroy(g.second);
        cudaEventDestroy(g.first);
    }
    for (void* p : b->old_host) cudaFreeHost(p);
    if (b->h_items) cudaFreeHost(b->h_items);
    if (b->items_staged) cudaEventDestroy(b->items_staged);
    if (b->setup) cudaStreamDestroy(b->setup);
    if (b->h_runs) cudaFreeHost(b->h_runs);
    if (b->staged) cudaEventDestroy(b->staged);
    b->timer.release();
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char* ecris_batch_last_error(const ecris_batch* b)
{
    return b ? b->err.c_str() : g_create_error.c_str();
}

ecris_status ecris_batch_add_run(ecris_batch* b, const ecris_geometry* geo, const ecris_bfield* bf,
                                 const ecris_grid* grid, const ecris_species* sp, const ecris_mcc* mcc,
                                 size_t n, const float* const xyzv[6], const uint8_t* q, double weight,
                                 uint64_t seed, double dt, int src_is_device, int32_t* run_out)
{
    if (!b) return ECRIS_EINVAL;
    if (!run_out || !grid || !mcc) return bfail(b, ECRIS_EINVAL, "batch_add_run: NULL argument");
    if (!finite_pos(dt)) return bfail(b, ECRIS_EINVAL, "batch_add_run: dt must be finite and > 0");
    const size_t need = ecris_run_bytes(n, grid->nx, grid->ny, grid->nz, (mcc->flags & kFCoulomb) != 0);
    if (b->budget && b->used + need > b->budget)
        return bfail(b, ECRIS_ENOMEM, "batch_add_run: the run (" + std::to_string(need) + " bytes) would exceed the "
                     "memory budget (" + std::to_string(b->used) + " of " + std::to_string(b->budget) + " used)");
    BCK(cudaSetDevice(b->device));
    batch_reap(b);
    // set the run up on the setup stream (its waits then cover only its own
    // copies), then hand it to the batch stream
    ecris_ctx* c = nullptr;
    ecris_status st = ecris_create(&c, b->device, b->setup);
    if (st != ECRIS_OK) return bfail(b, st, std::string("batch_add_run: ") + ecris_last_error(nullptr));
    st = ecris_init_fields(c, geo, bf, grid, sp, mcc);
    if (st == ECRIS_OK) st = ecris_load_ions(c, n, xyzv, q, weight, seed, src_is_device);
    if (st == ECRIS_OK) st = upload_dt(c, dt);
    if (st == ECRIS_OK && cudaStreamSynchronize(b->setup) != cudaSuccess) {
        st = ECRIS_ECUDA;
        c->err = "setup stream failed";
    }
    if (st != ECRIS_OK) {
        const std::string m = c->err;
        ecris_destroy(c);
        return bfail(b, st, "batch_add_run: " + m);
    }
    c->stream = b->stream;
    c->sort_every = b->sort_every;
    c->since_sort = c->sort_every;   // a batch run is grouped before its first step
    int32_t h = -1;
    for (size_t r = 0; r < b->runs.size(); ++r)
        if (!b->runs[r]) {
            h = (int32_t)r;
            break;
        }
    if (h < 0) {
        h = (int32_t)b->runs.size();
        b->runs.push_back(nullptr);
        b->bytes.push_back(0);
        b->dt.push_back(0.0);
    }
    b->runs[h] = c;
    b->bytes[h] = need;
    b->dt[h] = dt;
    b->used += need;
    b->layout_dirty = b->params_dirty = true;
    *run_out = h;
    return ECRIS_OK;
}

ecris_status ecris_batch_remove_run(ecris_batch* b, int32_t run)
{
    if (!b) return ECRIS_EINVAL;
    if (!run_live(b, run)) return bfail(b, ECRIS_EINVAL, "batch_remove_run: no such run");
    BCK(cudaSetDevice(b->device));
    batch_release_run(b, b->runs[run]);
    b->runs[run] = nullptr;
    b->used -= b->bytes[run];
    b->bytes[run] = 0;
    b->layout_dirty = b->params_dirty = true;
    return ECRIS_OK;
}

ecris_status ecris_batch_step(ecris_batch* b, uint32_t nsteps)
{
    if (!b) return ECRIS_EINVAL;
    BCK(cudaSetDevice(b->device));
    batch_reap(b);
    for (auto* c : b->runs)
        if (c && (c->failed || c->steps_done + nsteps >= kMaxSteps))
            return bfail(b, ECRIS_ESTATE, "batch_step: a run failed earlier or would pass 2^30 steps");
    if (b->layout_dirty) {
        ecris_status st = batch_items(b);
        if (st != ECRIS_OK) return st;
    }
    for (uint32_t s = 0; s < nsteps; ++s) {
        // regroup the particles of the runs that are due; their parameter
        // blocks change (the arrays swap), and so does the captured graph
        // when a run's collision kernels take the block by value
        // (several at once: the runs' sorts go to the side streams, whose
        // work the batch stream then waits for; timed steps sort one by one)
        int nsort = 0;
        for (auto* c : b->runs) {
            if (!c || c->n4 == 0 || c->since_sort < c->sort_every) continue;
            ecris_status st = ECRIS_OK;
            if (b->timer.on) {
                BCK(b->timer.run(kKindOther, b->stream, [&] {
                    st = sort_particles(c);
                    return cudaSuccess;
                }, 6));
            } else {
                const int k = nsort % kBatchSideStreams;
                if (nsort == 0) {
                    BCK(batch_side_streams(b));
                    BCK(cudaEventRecord(b->sort_fork, b->stream));
                }
                if (nsort < kBatchSideStreams) BCK(cudaStreamWaitEvent(b->side[k], b->sort_fork, 0));
                c->stream = b->side[k];
                st = sort_particles(c);
                c->stream = b->stream;
                ++nsort;
            }
            if (st != ECRIS_OK) return bfail(b, st, "batch_step: " + c->err);
            b->params_dirty = true;
            if (c->h.mcc.flags & kFCoulomb) b->graph_dirty = true;
        }
        for (int k = 0; k < nsort && k < kBatchSideStreams; ++k) {
            BCK(cudaEventRecord(b->sort_join[k], b->side[k]));
            BCK(cudaStreamWaitEvent(b->stream, b->sort_join[k], 0));
        }
        if (b->params_dirty) {
            ecris_status st = batch_upload(b);
            if (st != ECRIS_OK) return st;
        }
        if (!b->timer.on) {
            ecris_status st = batch_graph(b);
            if (st != ECRIS_OK) return st;
            BCK(cudaGraphLaunch(b->gexec, b->stream));
        } else {
            // timed: the same launches as the graph, one by one
            BCK(b->timer.run(kKindStep, b->stream, [&] {
                return launch_step_batch(b->d_runs, b->d_items, b->nitems, b->sm_count * batch_bps(b),
                                         b->variants, b->shape, b->stream);
            }));
            BCK(b->timer.run(kKindOther, b->stream, [&] {
                return launch_leave_batch(b->d_runs, (uint32_t)b->runs.size(), b->d_ticket, b->stream);
            }));
            for (auto* c : b->runs) {
                if (!c || !(c->h.mcc.flags & kFCoulomb)) continue;
                const uint32_t nc = (uint32_t)((size_t)c->h.nx * c->h.ny * c->h.nz);
                BCK(b->timer.run(kKindCoulomb, b->stream, [&] {
                    return launch_coulomb(*c->h_run, nc, c->btiles, c->d_ticket, c->collide_grid, 0u, 0, b->stream);
                }, kCoulombKernels));
            }
        }
        for (size_t r = 0; r < b->runs.size(); ++r) {
            ecris_ctx* c = b->runs[r];
            if (!c) continue;
            c->steps_done += 1;
            c->time_s += b->dt[r];
            ++c->since_sort;
            if (++c->since_fold >= c->fold_every) {
                const uint32_t nc = (uint32_t)((size_t)c->h.nx * c->h.ny * c->h.nz);
                BCK(b->timer.run(kKindOther, b->stream, [&] {
                    return launch_fold(*c->h_run, nc, c->d_count, c->d_charge, b->stream);
                }));
                c->since_fold = 0;
            }
        }
    }
    return ECRIS_OK;
}

ecris_status ecris_batch_diag(ecris_batch* b, int32_t run, ecris_diag_out* out)
{
    if (!b) return ECRIS_EINVAL;
    if (!run_live(b, run)) return bfail(b, ECRIS_EINVAL, "batch_diag: no such run");
    ecris_status st = ecris_diag(b->runs[run], out);
    if (st != ECRIS_OK) return bfail(b, st, "batch_diag: " + b->runs[run]->err);
    return ECRIS_OK;
}

ecris_status ecris_batch_update_ne(ecris_batch* b, int32_t run)
{
    if (!b) return ECRIS_EINVAL;
    if (!run_live(b, run)) return bfail(b, ECRIS_EINVAL, "batch_update_ne: no such run");
    BCK(cudaSetDevice(b->device));
    ecris_ctx* c = b->runs[run];
    if (c->failed) return bfail(b, ECRIS_ESTATE, "batch_update_ne: the run failed earlier");
    // the run's stream is the batch stream: the update follows the queued
    // steps.  Only the first update changes the parameter block (its gate)
    RunDev before;
    std::memcpy(&before, c->h_run, sizeof before);
    ecris_status st = update_ne(c);
    if (st == ECRIS_OK) st = upload_dt(c, b->dt[run]);
    if (st != ECRIS_OK) return bfail(b, st, "batch_update_ne: " + c->err);
    if (std::memcmp(&before, c->h_run, sizeof before) != 0) {
        b->params_dirty = true;
        if (c->h.mcc.flags & kFCoulomb) b->graph_dirty = true;
    }
    return ECRIS_OK;
}

ecris_status ecris_batch_get_fptd(ecris_batch* b, int32_t run, uint64_t* hist, uint64_t* age_sum)
{
    if (!b) return ECRIS_EINVAL;
    if (!run_live(b, run)) return bfail(b, ECRIS_EINVAL, "batch_get_fptd: no such run");
    BCK(cudaSetDevice(b->device));
    ecris_status st = get_fptd(b->runs[run], hist, age_sum);
    if (st != ECRIS_OK) return bfail(b, st, "batch_get_fptd: " + b->runs[run]->err);
    return ECRIS_OK;
}

ecris_status ecris_batch_get_extraction_radius(ecris_batch* b, int32_t run, double* r_sum)
{
    if (!b) return ECRIS_EINVAL;
    if (!run_live(b, run) || !r_sum) return bfail(b, ECRIS_EINVAL, "batch_get_extraction_radius: no such run");
    BCK(cudaSetDevice(b->device));
    ecris_status st = get_extraction_radius(b->runs[run], r_sum);
    if (st != ECRIS_OK) return bfail(b, st, "batch_get_extraction_radius: " + b->runs[run]->err);
    return ECRIS_OK;
}

ecris_status ecris_batch_set_probes(ecris_batch* b, int32_t run, const ecris_probe_spec* spec)
{
    if (!b) return ECRIS_EINVAL;
    if (!run_live(b, run) || !spec) return bfail(b, ECRIS_EINVAL, "batch_set_probes: no such run or no spec");
    BCK(cudaSetDevice(b->device));
    ecris_status st = set_probes(b->runs[run], spec);
    if (st != ECRIS_OK) return bfail(b, st, "batch_set_probes: " + b->runs[run]->err);
    return ECRIS_OK;
}

ecris_status ecris_batch_probe_sample(ecris_batch* b, int32_t run)
{
    if (!b) return ECRIS_EINVAL;
    if (!run_live(b, run)) return bfail(b, ECRIS_EINVAL, "batch_probe_sample: no such run");
    BCK(cudaSetDevice(b->device));
    ecris_status st = probe_sample(b->runs[run]);
    if (st != ECRIS_OK) return bfail(b, st, "batch_probe_sample: " + b->runs[run]->err);
    return ECRIS_OK;
}

ecris_status ecris_batch_get_probes(ecris_batch* b, int32_t run, uint64_t* samples, double* moments,
                                    uint64_t* screens)
{
    if (!b) return ECRIS_EINVAL;
    if (!run_live(b, run)) return bfail(b, ECRIS_EINVAL, "batch_get_probes: no such run");
    BCK(cudaSetDevice(b->device));
    ecris_status st = get_probes(b->runs[run], samples, moments, screens);
    if (st != ECRIS_OK) return bfail(b, st, "batch_get_probes: " + b->runs[run]->err);
    return ECRIS_OK;
}

ecris_status ecris_batch_get_cells(ecris_batch* b, int32_t run, float* ne, float* delta_x, float* delta_y)
{
    if (!b) return ECRIS_EINVAL;
    if (!run_live(b, run)) return bfail(b, ECRIS_EINVAL, "batch_get_cells: no such run");
    BCK(cudaSetDevice(b->device));
    ecris_status st = get_cells(b->runs[run], ne, delta_x, delta_y);
    if (st != ECRIS_OK) return bfail(b, st, "batch_get_cells: " + b->runs[run]->err);
    return ECRIS_OK;
}

ecris_status ecris_batch_get_state(ecris_batch* b, int32_t run, float* const xyzv[6], uint32_t* meta,
                                   int dst_is_device)
{
    if (!b) return ECRIS_EINVAL;
    if (!run_live(b, run)) return bfail(b, ECRIS_EINVAL, "batch_get_state: no such run");
    ecris_status st = ecris_get_state(b->runs[run], xyzv, meta, dst_is_device);
    if (st != ECRIS_OK) return bfail(b, st, "batch_get_state: " + b->runs[run]->err);
    return ECRIS_OK;
}

ecris_status ecris_batch_memory(const ecris_batch* b, size_t* used, size_t* budget)
{
    if (!b) return ECRIS_EINVAL;
    if (used) *used = b->used;
    if (budget) *budget = b->budget;
    return ECRIS_OK;
}

ecris_status ecris_batch_set_profiling(ecris_batch* b, int enable)
{
    if (!b) return ECRIS_EINVAL;
    BCK(cudaSetDevice(b->device));
    BCK(b->timer.collect(b->stream));
    b->timer.reset(enable != 0);
    return ECRIS_OK;
}

ecris_status ecris_batch_get_profile(ecris_batch* b, ecris_profile* out)
{
    if (!b) return ECRIS_EINVAL;
    if (!out) return bfail(b, ECRIS_EINVAL, "batch_get_profile: out is NULL");
    BCK(cudaSetDevice(b->device));
    BCK(b->timer.collect(b->stream));
    b->timer.fill(out);
    return ECRIS_OK;
}

ecris_status ecris_batch_set_tuning(ecris_batch* b, const ecris_tuning* t)
{
    if (!b) return ECRIS_EINVAL;
    if (!t) return bfail(b, ECRIS_EINVAL, "batch_set_tuning: NULL argument");
    if (t->sort_every < 1 || t->blocks_per_sm < 0)
        return bfail(b, ECRIS_EINVAL, "batch_set_tuning: need sort_every >= 1 and blocks_per_sm >= 0");
    int shape = -1;
    if (t->threads == 0 && t->particles_per_thread == 0 && t->stages >= 0 && t->stages <= 3 && t->stages != 1)
        shape = t->stages == 2 ? 4 : kDefaultShape;   // 256 x 2 with two or three stages
    // stages 0: the three-stage form where the shape has one
    for (int k = 0; k < kStepShapes; ++k)
        if (t->threads == kShapeThreads[k] && t->particles_per_thread == kShapeVec[k] &&
            (t->stages == kShapeStages[k] || (t->stages == 0 && (shape < 0 || kShapeStages[k] == 3))))
            shape = k;
    if (shape < 0)
        return bfail(b, ECRIS_EINVAL,
                     "batch_set_tuning: threads must be 128, 256 or 512, particles_per_thread 1, 2 or 4 and "
                     "stages 2, or 3 for 128 x 2, 256 x 1 and 256 x 2 (all 0: 256 x 2 x 3)");
    b->sort_every = (uint32_t)t->sort_every;
    for (auto* c : b->runs)
        if (c) {
            c->sort_every = b->sort_every;
            if (c->since_sort > c->sort_every) c->since_sort = c->sort_every;
        }
    b->blocks_per_sm = t->blocks_per_sm;
    if (shape != b->shape) {
        b->shape = shape;
        b->layout_dirty = true;   // the runs' tiles and the work list change with the tile size
    }
    b->graph_dirty = true;
    return ECRIS_OK;
}

}  // extern "C"

namespace {

// Everything a step of a batch run changes, copied aside so that the
// autotuner's trial steps can be undone: the current particle set, the
// tallies, deposit and time sums, first-passage records, step counter and
// error word on the device, and the host's step bookkeeping.
struct RunSnapshot {
    unsigned char* buf = nullptr;
    size_t bytes = 0;
    uint64_t steps_done = 0;
    double time_s = 0.0;
    uint32_t since_sort = 0, since_fold = 0, calls_since_load = 0;
};

template <class F>
void snapshot_parts(ecris_ctx* c, F f)
{
    const size_t cap = c->cap, nc = c->cap_cells;
    for (int k = 0; k < 6; ++k) f((void*)c->d_soa[k], cap * 4);
    f((void*)c->d_meta, cap * 4);
    f((void*)c->d_id, cap * 4);
    f((void*)c->d_tally, kTallyWords * sizeof(unsigned long long));
    f((void*)c->d_dep, nc * sizeof(unsigned long long));
    f((void*)c->d_count, nc * sizeof(unsigned long long));
    f((void*)c->d_charge, nc * sizeof(unsigned long long));
    f((void*)c->d_birth, cap * 4);
    f((void*)c->d_fptd, kFptdWords * sizeof(unsigned long long));
    f((void*)c->d_step, sizeof(uint32_t));
    f((void*)c->d_err, sizeof(uint32_t));
}

ecris_status snapshot_take(ecris_batch* b, ecris_ctx* c, RunSnapshot& sn)
{
    size_t total = 0;
    snapshot_parts(c, [&](void*, size_t n) { total += (n + 255) & ~(size_t)255; });
    BCK(cudaMallocAsync((void**)&sn.buf, total, b->stream));
    sn.bytes = total;
    size_t off = 0;
    cudaError_t e = cudaSuccess;
    snapshot_parts(c, [&](void* p, size_t n) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(sn.buf + off, p, n, cudaMemcpyDeviceToDevice, b->stream);
        off += (n + 255) & ~(size_t)255;
    });
    BCK(e);
    sn.steps_done = c->steps_done;
    sn.time_s = c->time_s;
    sn.since_sort = c->since_sort;
    sn.since_fold = c->since_fold;
    sn.calls_since_load = c->calls_since_load;
    return ECRIS_OK;
}

// copy back into the run's current particle set (a sort may have swapped the
// sets since: the copies go wherever the arrays now are)
ecris_status snapshot_restore(ecris_batch* b, ecris_ctx* c, RunSnapshot& sn)
{
    size_t off = 0;
    cudaError_t e = cudaSuccess;
    snapshot_parts(c, [&](void* p, size_t n) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(p, sn.buf + off, n, cudaMemcpyDeviceToDevice, b->stream);
        off += (n + 255) & ~(size_t)255;
    });
    BCK(e);
    BCK(cudaFreeAsync(sn.buf, b->stream));
    sn.buf = nullptr;
    c->steps_done = sn.steps_done;
    c->time_s = sn.time_s;
    c->since_sort = sn.since_sort;
    c->since_fold = sn.since_fold;
    c->calls_since_load = sn.calls_since_load;
    return ECRIS_OK;
}

// time per step of `steps` steps of the batch in its current tuning, with
// no sort among them (hold = true) or in whole sort periods starting with a
// sort; one untimed step first takes the graph capture out of the timing
ecris_status time_steps(ecris_batch* b, uint32_t steps, bool hold, float* ms_per_step)
{
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    BCK(cudaEventCreate(&t0));
    BCK(cudaEventCreate(&t1));
    const uint32_t keep = b->sort_every;
    auto set_sort = [&](uint32_t every, bool due) {
        for (auto* c : b->runs)
            if (c) {
                c->sort_every = every;
                c->since_sort = due ? every : 0u;
            }
    };
    if (hold) set_sort(0xFFFFFFFFu, false);
    ecris_status st = ecris_batch_step(b, 1);
    if (st == ECRIS_OK) {
        if (!hold) set_sort(keep, true);
        cudaEventRecord(t0, b->stream);
        st = ecris_batch_step(b, steps);
        cudaEventRecord(t1, b->stream);
    }
    if (cudaEventSynchronize(t1) != cudaSuccess && st == ECRIS_OK) st = ECRIS_ECUDA;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, t0, t1);
    *ms_per_step = ms / (float)(steps ? steps : 1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    set_sort(keep, false);
    return st;
}

}  // namespace

extern "C" {

ecris_status ecris_batch_autotune(ecris_batch* b, uint32_t trial_steps, ecris_tuning* chosen)
{
    return ecris::batch_autotune(b, trial_steps, true, chosen);
}

}  // extern "C"

namespace ecris {

ecris_status batch_autotune(ecris_batch* b, uint32_t trial_steps, bool cadence, ecris_tuning* chosen)
{
    if (!b) return ECRIS_EINVAL;
    BCK(cudaSetDevice(b->device));
    if (trial_steps < 1) trial_steps = 1;
    // the runs' state before the trials, restored afterwards
    std::vector<RunSnapshot> snaps(b->runs.size());
    ecris_status st = ECRIS_OK;
    for (size_t r = 0; r < b->runs.size() && st == ECRIS_OK; ++r)
        if (b->runs[r]) st = snapshot_take(b, b->runs[r], snaps[r]);
    const int orig_shape = b->shape, orig_bps = b->blocks_per_sm;
    const uint32_t orig_sort = b->sort_every;
    // the trials run on the grouped layout: every run is sorted first (the
    // state is restored afterwards anyway)
    for (auto* c : b->runs)
        if (c) c->since_sort = c->sort_every;
    if (st == ECRIS_OK) st = ecris_batch_step(b, 1);
    int best_shape = orig_shape, best_bps = orig_bps;
    uint32_t best_sort = orig_sort;
    float best = 1e30f, ms = 0.0f;
    auto apply = [&](int shape, int bps, uint32_t every) {
        if (shape != b->shape) b->layout_dirty = true;
        b->shape = shape;
        b->blocks_per_sm = bps;
        b->sort_every = every;
        b->graph_dirty = true;
    };
    // 1. the launch shape (threads per block x particles per thread), as many
    // resident blocks as fit, no sorts among the timed steps
    for (int k = 0; k < kStepShapes && st == ECRIS_OK; ++k) {
        apply(k, 0, orig_sort);
        st = time_steps(b, trial_steps, true, &ms);
        if (st == ECRIS_OK && ms < best) {
            best = ms;
            best_shape = k;
        }
    }
    // 2. resident blocks per SM of that shape
    best = 1e30f;
    for (int bps = 1; bps <= b->max_bps[best_shape] && st == ECRIS_OK; ++bps) {
        apply(best_shape, bps, orig_sort);
        st = time_steps(b, trial_steps, true, &ms);
        if (st == ECRIS_OK && ms < best) {
            best = ms;
            best_bps = bps;
        }
    }
    // 3. steps between sorts: whole sort periods, each starting with a sort,
    // so that every cadence pays its own share of sorting
    best = 1e30f;
    const uint32_t cadences[5] = {8, 32, 128, 256, 512};
    for (int k = 0; k < 5 && st == ECRIS_OK && cadence; ++k) {
        apply(best_shape, best_bps, cadences[k]);
        const uint32_t steps = ((trial_steps + cadences[k] - 1) / cadences[k]) * cadences[k];
        st = time_steps(b, steps, false, &ms);
        if (st == ECRIS_OK && ms < best) {
            best = ms;
            best_sort = cadences[k];
        }
    }
    // undo the trial steps
    for (size_t r = 0; r < b->runs.size(); ++r)
        if (b->runs[r] && snaps[r].buf) {
            const ecris_status s2 = snapshot_restore(b, b->runs[r], snaps[r]);
            if (st == ECRIS_OK) st = s2;
        }
    if (st != ECRIS_OK) {
        apply(orig_shape, orig_bps, orig_sort);
        for (auto* c : b->runs)
            if (c) {
                c->sort_every = orig_sort;
                c->since_sort = orig_sort;
            }
        return st;
    }
    apply(best_shape, best_bps, best_sort);
    // the restored particles are in the order they had before the trials:
    // every run regroups at its next step (the layout changes no result)
    for (auto* c : b->runs)
        if (c) {
            c->sort_every = best_sort;
            c->since_sort = best_sort;
        }
    if (chosen) {
        std::memset(chosen, 0, sizeof *chosen);
        chosen->sort_every = (int32_t)best_sort;
        chosen->blocks_per_sm = best_bps;
        chosen->threads = kShapeThreads[best_shape];
        chosen->particles_per_thread = kShapeVec[best_shape];
        chosen->stages = kShapeStages[best_shape];
    }
    return ECRIS_OK;
}

}  // namespace ecris

extern "C" {

}  // extern "C"

// ---------------------------------------------------------------------------
// Hooks of the served form
// ---------------------------------------------------------------------------
namespace ecris {

const float* nanbu_table()
{
    // the same for every run: built once per process
    static const std::vector<float> t = [] {
        std::vector<float> v(kNanbuN);
        const double l0 = std::log(kNanbuSLo), dl = std::log(kNanbuSHi / kNanbuSLo) / (kNanbuN - 1);
        for (int i = 0; i < kNanbuN; ++i) v[i] = (float)std::log(nanbu_A_host(std::exp(l0 + i * dl)));
        return v;
    }();
    return t.data();
}

float coulomb_s_coef(double lnL_ii, double mass_amu, double weight, double cell_volume_m3)
{
    const double mu = 0.5 * mass_amu * kAmu;
    const double k = kE * kE / (kEps0 * mu);
    return (float)(lnL_ii / (4.0 * kPi) * k * k * weight / cell_volume_m3);
}

ecris_status batch_snapshot(ecris_batch* b, int32_t run, TallySnapshot* dst)
{
    if (!run_live(b, run)) return bfail(b, ECRIS_EINVAL, "batch_snapshot: no such run");
    const ecris_ctx* c = b->runs[run];
    BCK(cudaMemcpyAsync(dst->tally, c->d_tally, sizeof dst->tally, cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaMemcpyAsync(&dst->err, c->d_err, sizeof dst->err, cudaMemcpyDeviceToHost, b->stream));
    return ECRIS_OK;
}

cudaStream_t batch_stream(const ecris_batch* b) { return b->stream; }

void batch_snapshot_diag(const ecris_batch* b, int32_t run, const TallySnapshot& snap, uint64_t steps,
                         ecris_diag_out* out)
{
    const ecris_ctx* c = b->runs[run];
    fill_diag(c->h, c->weight, snap.tally, nullptr, steps, (double)steps * b->dt[run], out);
}

}  // namespace ecris
