// Fused per-macroparticle time step (push -> boundary test -> MCC -> NGP
// deposition) of the ECRIS model of Mironov et al. (arXiv:1507.03392, Sec.
// II), the wall and aperture bookkeeping of the particles that left the
// chamber in the step, the deposit fold and the charge-state census used by
// the diagnostics, and the cell-count scan that starts the Coulomb collisions
// (which, in a one-run step, also runs the leaver pass in extra blocks).
//
// Data layout: each run's particles are SoA arrays x, y, z (fixed point), vx,
// vy, vz, a u32 meta word and a u32 stable id, padded to a multiple of 4.
// The step kernel streams tiles of them through shared memory with the bulk
// copy engine.  Per-cell data (n_e, zone, delta) and the E grid are float4
// records read through L1/L2; the rate table is read through L1.  The deposit
// is one packed 64-bit reduction per run of lanes in the same cell (count in
// the high word, charge in the low word).  A particle that leaves the chamber
// is only listed by the step kernel; a second, small pass does its crossing
// geometry (FP64), tallies and re-emission, so the step kernel carries no
// FP64 code and no per-tile tally traffic.
#include "ecris_internal.cuh"

namespace ecris {

namespace {

// Cosine-law re-emission at temperature T0 (full accommodation): normal speed
// sigma sqrt(-2 ln U0) along the inward normal n, tangential components one
// Box-Muller pair along e1, e2.
__device__ __forceinline__ void emit(float sigma, float nx, float ny, float nz, float e1x, float e1y,
                                     float e1z, float e2x, float e2y, float e2z, const Words& w,
                                     float& vx, float& vy, float& vz)
{
    const float vn = sigma * sqrtf(-2.0f * logf(unit01(w.w0)));
    const float rt = sigma * sqrtf(-2.0f * logf(unit01(w.w1)));
    float s, c;
    sincospif(2.0f * unit01(w.w2), &s, &c);
    const float t1 = rt * c, t2 = rt * s;
    vx = vn * nx + t1 * e1x + t2 * e2x;
    vy = vn * ny + t1 * e1y + t2 * e2y;
    vz = vn * nz + t1 * e1z + t2 * e2z;
}

// |v|^2 + a, contraction written out
__device__ __forceinline__ float norm2_plus(float vx, float vy, float vz, float a)
{
    return fmaf(vx, vx, fmaf(vy, vy, fmaf(vz, vz, a)));
}

// probability 1 - exp(-lam) of at least one event in a step; for small lam
// the cubic Taylor polynomial is exact to FP32 rounding (error < lam^4 / 24)
__device__ __forceinline__ float event_prob(float lam)
{
    if (lam < 1e-3f) return lam * fmaf(-lam, fmaf(-lam, 1.0f / 6.0f, 0.5f), 1.0f);
    return -expm1f(-lam);
}

// 64-bit displacement for the rare step longer than 2^30 fixed-point units
// (kept out of line: the common path converts in 32 bits)
struct Disp { long long x, y, z; };

__device__ __noinline__ Disp far_displacement(float dx, float dy, float dz)
{
    return Disp{__float2ll_rn(fminf(fmaxf(dx, -1e12f), 1e12f)), __float2ll_rn(fminf(fmaxf(dy, -1e12f), 1e12f)),
                __float2ll_rn(fminf(fmaxf(dz, -1e12f), 1e12f))};
}

// Position after the step's straight move with the (already pushed)
// velocity, in 64-bit fixed point.  The step kernel and the leaver pass both
// call this, so they get the same integers.  The displacement is rounded to
// nearest; below 2^30 units a 32-bit conversion gives the same integer,
// larger (or non-finite) ones take the bounded 64-bit conversion.
__device__ __forceinline__ void displace(const RunDev& R, int32_t X, int32_t Y, int32_t Z, float vx, float vy,
                                         float vz, long long& xn, long long& yn, long long& zn)
{
    xn = X;
    yn = Y;
    zn = Z;
    if (!(R.flags & kFPush)) return;
    const float dx = vx * R.dt_sxy, dy = vy * R.dt_sxy, dz = vz * R.dt_sz;
    if (fmaxf(fabsf(dx), fmaxf(fabsf(dy), fabsf(dz))) < 1.0e9f) {
        xn += __float2int_rn(dx);
        yn += __float2int_rn(dy);
        zn += __float2int_rn(dz);
    } else {
        const Disp d = far_displacement(dx, dy, dz);
        xn += d.x;
        yn += d.y;
        zn += d.z;
    }
}

constexpr long long kLim = 2147483648ll;   // 2^31: the fixed-point range

// Boundary test on the new position, exact in fixed point: outside the
// cylinder wall (r > R0), behind the injection plane (z < 0), past the
// extraction plane (z >= L).
__device__ __forceinline__ void outside(long long xn, long long yn, long long zn, bool& out_r, bool& out_0,
                                        bool& out_L)
{
    const bool out_xy = xn < -kLim || xn >= kLim || yn < -kLim || yn >= kLim;
    out_r = out_xy || (long long)(int32_t)xn * (int32_t)xn + (long long)(int32_t)yn * (int32_t)yn > (1ll << 62);
    out_0 = zn < -kLim;
    out_L = zn >= kLim;
}

__device__ __forceinline__ int32_t clamp_fx(long long v) { return (int32_t)max(min(v, kLim - 1), -kLim); }

// a + b in 32 bits, and whether the exact sum left the 32-bit range
__device__ __forceinline__ int32_t add_wrap(int32_t a, int32_t b, bool& over)
{
    const int32_t s = (int32_t)((uint32_t)a + (uint32_t)b);
    over = ((a ^ s) & (b ^ s)) < 0;
    return s;
}

// The straight move of the step and the boundary test, as displace() and
// outside() give them, but in 32-bit arithmetic for the common step shorter
// than 2^30 units: the fixed-point range is the chamber's bounding box, so a
// sum that leaves the 32-bit range has left the chamber.  On return X, Y, Z
// hold the new position (clamped into the range for a leaver); true if the
// particle left.
__device__ __forceinline__ bool move(const RunDev& R, int32_t& X, int32_t& Y, int32_t& Z, float vx, float vy,
                                     float vz)
{
    const bool push = (R.flags & kFPush) != 0;
    const float dx = push ? vx * R.dt_sxy : 0.0f, dy = push ? vy * R.dt_sxy : 0.0f, dz = push ? vz * R.dt_sz : 0.0f;
    if (fmaxf(fabsf(dx), fmaxf(fabsf(dy), fabsf(dz))) < 1.0e9f) {
        bool ox, oy, oz;
        const int32_t xn = add_wrap(X, __float2int_rn(dx), ox);
        const int32_t yn = add_wrap(Y, __float2int_rn(dy), oy);
        const int32_t zn = add_wrap(Z, __float2int_rn(dz), oz);
        const bool leave = ox | oy | oz ||
                           (long long)xn * xn + (long long)yn * yn > (1ll << 62);
        if (!leave) {
            X = xn;
            Y = yn;
            Z = zn;
        }
        return leave;
    }
    long long xn, yn, zn;
    displace(R, X, Y, Z, vx, vy, vz, xn, yn, zn);
    bool out_r, out_0, out_L;
    outside(xn, yn, zn, out_r, out_0, out_L);
    if (out_r | out_0 | out_L) return true;
    X = clamp_fx(xn);
    Y = clamp_fx(yn);
    Z = clamp_fx(zn);
    return false;
}

// Elastic ion-atom scattering (a rare event, kept out of line so that the
// per-particle code's registers do not carry it): isotropic in the
// centre-of-mass frame with a background atom drawn at T0 from the stream-3
// words u; the new direction of the relative velocity from the wall stream,
// unused by a particle that stays inside
__device__ __noinline__ void elastic_scatter(const RunDev& R, const Words& u, uint32_t pid, uint32_t step, float& vx,
                                             float& vy, float& vz)
{
    const Words d = rng_words(R, pid, step, 2u);
    float s1, c1, s2, c2;
    const float r1 = R.sig0 * sqrtf(-2.0f * logf(unit01(u.w0)));
    sincospif(2.0f * unit01(u.w1), &s1, &c1);
    const float r2 = R.sig0 * sqrtf(-2.0f * logf(unit01(u.w2)));
    sincospif(2.0f * unit01(u.w3), &s2, &c2);
    const float ax = r1 * c1, ay = r1 * s1, az = r2 * c2;
    const float gx = vx - ax, gy = vy - ay, gz = vz - az;
    const float gm = sqrtf(gx * gx + gy * gy + gz * gz);
    const float ct = 2.0f * unit01(d.w0) - 1.0f;
    const float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
    float sp, cp;
    sincospif(2.0f * unit01(d.w1), &sp, &cp);
    vx = 0.5f * (vx + ax) + 0.5f * gm * (st * cp);
    vy = 0.5f * (vy + ay) + 0.5f * gm * (st * sp);
    vz = 0.5f * (vz + az) + 0.5f * gm * ct;
}

// false if no cell can ionise an atom whose ionisation word is w0: the gate
// bounds the threshold of every cell.  It comes with the parameter block
// while the host knows the densest cell, else from the word the device keeps
// after the rate table (a gate of 0 reads the same either way)
__device__ __forceinline__ bool atom_may_ionize(const RunDev& R, uint32_t w0)
{
    uint32_t gate = R.atom_gate;
    if (gate == 0u) gate = __ldg(reinterpret_cast<const uint32_t*>(R.kdt) + kGateWord);
    return w0 < gate || gate == 0xFFFFFFFFu;
}

// Advance one particle by one step.  pid is its stable id (the Philox counter
// word).  On return dep_cell is the cell it deposits in and ckey the cell
// where it takes part in Coulomb collisions (kNoCell if it does not).  A
// particle that left the chamber keeps its old position and returns true
// with its pushed velocity: the leaver pass finishes its step.
// kVar: with the code of the opt-in processes (double ionisation, elastic
// ion-atom scattering); without it the kernels carry none of their branches
template <bool kVar>
__device__ __forceinline__ bool step_particle(const RunDev& R, uint32_t pid, uint32_t step, int32_t& X,
                                              int32_t& Y, int32_t& Z, float& vx, float& vy, float& vz,
                                              uint32_t& meta, uint32_t& ckey, uint32_t& dep_cell)
{
    ckey = kNoCell;
    dep_cell = kNoCell;
    const uint32_t status = meta & 0xFFFF0000u;
    if (status & (kStFrozen | kStPad)) {
        meta = status | (meta & kQMask);   // events of a frozen particle are cleared
        return false;
    }
    uint32_t Q = meta & kQMask;
    uint32_t ev = 0;

    // ---- push: Boris rotation for ions, straight line for atoms ----
    // an ion's cell record is fetched with its field gather, at the old
    // position; the push moves it far less than a cell, so it is reused
    // unless the particle crossed into another cell
    uint32_t cell_pre = kNoCell;
    float4 cr = make_float4(0.f, 0.f, 0.f, 0.f);
    if (Q > 0) {
        cell_pre = ngp_cell(R, X, Y, Z);
        cr = __ldg(R.cell + cell_pre);
    }
    if ((R.flags & kFPush) && Q > 0) {
        const float x0 = fx_xy(R, X), y0 = fx_xy(R, Y), z0 = fx_z(R, Z);
        float Bx, By, Bz, Ex, Ey, Ez;
        if (kVar && R.btab) bfield_table(R, x0, y0, z0, Bx, By, Bz);
        else bfield(R, x0, y0, z0, Bx, By, Bz);
        if (R.flags & kFHasE) {
            efield(R, x0, y0, z0, Ex, Ey, Ez);
        } else {
            Ex = 0.0f;   // no E grid: the gather would return zeros
            Ey = 0.0f;
            Ez = 0.0f;
        }
        // (FMAs written out: this file is compiled without contraction)
        const float h = (float)Q * R.qm_unit * R.half_dt;
        float mx = fmaf(h, Ex, vx), my = fmaf(h, Ey, vy), mz = fmaf(h, Ez, vz);
        const float tx = h * Bx, ty = h * By, tz = h * Bz;
        const float sf = __fdividef(2.0f, fmaf(tx, tx, fmaf(ty, ty, fmaf(tz, tz, 1.0f))));
        const float px = mx + fmaf(my, tz, -mz * ty);
        const float py = my + fmaf(mz, tx, -mx * tz);
        const float pz = mz + fmaf(mx, ty, -my * tx);
        mx = fmaf(fmaf(py, tz, -pz * ty), sf, mx);
        my = fmaf(fmaf(pz, tx, -px * tz), sf, my);
        mz = fmaf(fmaf(px, ty, -py * tx), sf, mz);
        vx = fmaf(h, Ex, mx);
        vy = fmaf(h, Ey, my);
        vz = fmaf(h, Ez, mz);
    }
    const int32_t X0 = X, Y0 = Y, Z0 = Z;
    if (move(R, X, Y, Z, vx, vy, vz)) {
        X = X0;   // the leaver pass redoes the move from the old position
        Y = Y0;
        Z = Z0;
        meta = status | Q;
        return true;
    }

    // ---- MCC in the particle's cell ----
    const uint32_t cell = ngp_cell(R, X, Y, Z);
    const Words w = rng_words(R, pid, step, 0u);
    // an atom needs its cell only if its ionisation word could fire in
    // the densest cell; otherwise no cell can ionise it this step
    const bool ionize = (R.flags & kFIonize) && (int)Q < R.qmax;
    const bool need = Q > 0 || (ionize && atom_may_ionize(R, w.w0));
    if (need && cell != cell_pre) cr = __ldg(R.cell + cell);   // n_e, zone, delta_x, delta_y
    const int zone = cr.y > 0.5f ? 1 : 0;
    const bool recomb = kVar && (R.flags & kFRecomb) && Q >= 1;
    if ((ionize && need) || recomb) {
        const float lam = cr.x * __ldg(R.kdt + zone * kQSlots + Q);
        if constexpr (kVar) {
            const float p = event_prob(lam);
            if (fires(w.w0, p)) {
                // single, double, triple and recombination share [0, p) in
                // proportion to their rates: below p k1/k one electron goes,
                // below p (k1+k2)/k two, below p (k1+k2+k3)/k three, above
                // that one is captured
                int up = 1;
                if (R.flags & (kFDouble | kFRecomb)) {
                    if (!fires(w.w0, p * __ldg(R.kdt + 2 * kQSlots + zone * kQSlots + Q))) {
                        if (fires(w.w0, p * __ldg(R.kdt + 4 * kQSlots + zone * kQSlots + Q))) up = 2;
                        else up = fires(w.w0, p * __ldg(R.kdt + 6 * kQSlots + zone * kQSlots + Q)) ? 3 : -1;
                    }
                }
                if (up > 0) {
                    if (Q == 0) R.birth[pid] = step;   // an ion is born (first-passage clock)
                    Q += (uint32_t)up;
                    ev |= kEvIonize;
                } else {
                    Q -= 1u;
                    ev |= kEvRecomb;
                }
            }
        } else if (fires(w.w0, event_prob(lam))) {
            if (Q == 0) R.birth[pid] = step;   // an ion is born (first-passage clock)
            Q += 1;
            ev |= kEvIonize;
        }
    }
    // collisions with the neutral background: 1 charge exchange, 2 elastic
    uint32_t coll = 0u;
    if (kVar && (R.flags & kFElastic) && R.n0sel > 0.0f) {
        if (Q >= 1) {
            // either process with probability 1 - exp(-n0 (sigma_cx + sigma_el)
            // v_rel dt), shared in proportion to the cross sections
            const float vrel = sqrt_approx(norm2_plus(vx, vy, vz, R.vth2));
            const float scx = ((R.flags & kFCx) && Q != 2) ? R.n0s1 * (float)Q : 0.0f;
            const float sel = R.n0sel * (float)Q;
            const float pt = event_prob((scx + sel) * vrel * R.dt);
            if (fires(w.w1, pt)) coll = fires(w.w1, pt * (scx / (scx + sel))) ? 1u : 2u;
        }
    } else if ((R.flags & kFCx) && R.n0s1 > 0.0f && Q >= 1 && Q != 2) {
        const float vrel = sqrt_approx(norm2_plus(vx, vy, vz, R.vth2));
        const float p = event_prob(R.n0s1 * (float)Q * vrel * R.dt);
        if (fires(w.w1, p)) coll = 1u;
    }
    if (coll) {
        const Words u = rng_words(R, pid, step, 3u);
        if (kVar && coll == 2u) {
            elastic_scatter(R, u, pid, step, vx, vy, vz);
            ev |= kEvElastic;
        } else {
            ev |= kEvCx;
            if (Q == 1) {
                float s1, c1, s2, c2;
                const float r1 = R.sig0 * sqrtf(-2.0f * logf(unit01(u.w0)));
                sincospif(2.0f * unit01(u.w1), &s1, &c1);
                const float r2 = R.sig0 * sqrtf(-2.0f * logf(unit01(u.w2)));
                sincospif(2.0f * unit01(u.w3), &s2, &c2);
                vx = r1 * c1; vy = r1 * s1; vz = r2 * c2;
            } else {
                const float ct = 2.0f * unit01(u.w0) - 1.0f;
                const float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
                float sp, cp;
                sincospif(2.0f * unit01(u.w1), &sp, &cp);
                vx += R.dv_cx * st * cp;
                vy += R.dv_cx * st * sp;
                vz += R.dv_cx * ct;
                Q -= 1;
            }
        }
    }
    if ((R.flags & kFEikick) && Q >= 1) {
        const float qp = R.ei_pow == 1 ? (float)Q : (float)(Q * Q);
        const float D = sqrt_approx((zone ? R.ei_coef[1] : R.ei_coef[0]) * cr.x * qp);
        const float ct = fmaf(2.0f, unit01(w.w2), -1.0f);
        const float st = sqrt_approx(fmaxf(0.0f, fmaf(-ct, ct, 1.0f)));
        float sp, cp;
        sincos_2pi(unit01(w.w3), &sp, &cp);   // azimuth
        const float dxv = fmaf(st, cp, cr.z), dyv = fmaf(st, sp, cr.w), dzv = ct;
        const float m2 = norm2_plus(dxv, dyv, dzv, 0.0f);
        if (m2 > 0.0f) {
            const float k = D * rsqrtf(m2);
            vx = fmaf(k, dxv, vx);
            vy = fmaf(k, dyv, vy);
            vz = fmaf(k, dzv, vz);
        }
    }
    if (Q >= 1 && (R.flags & kFCoulomb)) ckey = cell;
    dep_cell = cell;   // NGP deposition at the final position (aggregated over the warp by the caller)
    meta = status | ev | Q;
    return false;
}

// first-passage time of an extracted ion, age in steps (>= 1 for an ion born
// in an earlier step): 4 log bins per octave, and the age summed by Q
__device__ __forceinline__ void fptd_record(const RunDev& R, uint32_t Q, uint32_t age)
{
    if (age == 0u) return;
    const int e = 31 - __clz(age);
    const uint32_t m = e >= 2 ? (age >> (e - 2)) & 3u : (age << (2 - e)) & 3u;
    atomicAdd(R.fptd + Q * kFptdBins + 4 * e + m, 1ull);
    atomicAdd(R.fptd + kFptdAgeSum + Q, (unsigned long long)age);
}

// Finish the step of a particle that left the chamber (the step kernel kept
// its old position X, Y, Z and its pushed velocity): the first crossing of
// the straight segment with the wall, the injection plane or the extraction
// plane, in FP64 from the exact fixed-point coordinates; the extracted / lost
// tallies and the energy carried to the wall; then re-emission (cosine law at
// T0 from the crossing point, or from the inlet after extraction) or, without
// recycling, freezing.  Returns the cell it deposits in (kNoCell if frozen).
__device__ __forceinline__ uint32_t leave_particle(const RunDev& R, uint32_t pid, uint32_t step, int32_t& X,
                                                   int32_t& Y, int32_t& Z, float& vx, float& vy, float& vz,
                                                   uint32_t& meta)
{
    const uint32_t status = meta & 0xFFFF0000u;
    const uint32_t Q = meta & kQMask;
    long long xn, yn, zn;
    displace(R, X, Y, Z, vx, vy, vz, xn, yn, zn);
    bool out_r, out_0, out_L;
    outside(xn, yn, zn, out_r, out_0, out_L);

    const double sxy = R.sxy_d, szd = R.sz_d;
    const double dx0 = (double)X * sxy, dy0 = (double)Y * sxy, dz0 = ((double)Z + 2147483648.0) * szd;
    const double ddx = (double)(xn - X) * sxy, ddy = (double)(yn - Y) * sxy, ddz = (double)(zn - Z) * szd;
    double fbest = 2.0;
    int kind = 0;
    if (out_r) {
        // |p0 + f d|^2 = R0^2 with c = |p0|^2 - R0^2 <= 0, taken exactly in fixed point
        const double a = ddx * ddx + ddy * ddy, b = dx0 * ddx + dy0 * ddy;
        const double c = (double)((long long)X * X + (long long)Y * Y - (1ll << 62)) * sxy * sxy;
        const double disc = sqrt(fmax(0.0, b * b - a * c));
        double f = (b + disc > 0.0) ? -c / (b + disc) : 0.0;
        f = fmax(f, 0.0);
        fbest = f;
        kind = 1;
    }
    if (out_0) {
        const double f = (double)((long long)Z + kLim) / (double)((long long)Z - zn);
        if (f < fbest) { fbest = f; kind = 2; }
    }
    if (out_L) {
        const double f = (double)(kLim - (long long)Z) / (double)(zn - (long long)Z);
        if (f < fbest) { fbest = f; kind = 3; }
    }
    const double cxd = dx0 + fbest * ddx, cyd = dy0 + fbest * ddy, czd = dz0 + fbest * ddz;
    if (kind == 3 && cxd * cxd + cyd * cyd < R.r_ap_d * R.r_ap_d) kind = 4;

    // ---- wall / aperture bookkeeping ----
    if (Q >= 1) atomicAdd(R.tally + kTallyKe, __float2ull_rn(R.ke_scale * (vx * vx + vy * vy + vz * vz)));
    uint32_t ev;
    if (kind == 4) {
        atomicAdd(R.tally + kTallyExtracted + Q, 1ull);
        ev = kEvExtract;
        const uint32_t born = Q >= 1 ? R.birth[pid] : 0xFFFFFFFFu;
        if (born <= step) fptd_record(R, Q, step - born);
        // radius at the aperture plane (mean radial displacement by Q), in nm
        atomicAdd(R.fptd + kFptdRadius + Q, (unsigned long long)rint(sqrt(cxd * cxd + cyd * cyd) * 1e9));
    } else {
        atomicAdd(R.tally + kTallyLost + Q, 1ull);
        ev = kEvWall;
    }
    if (!(R.flags & kFRecycle)) {
        // frozen at its last position, clamped into the fixed-point range
        X = clamp_fx(xn);
        Y = clamp_fx(yn);
        Z = clamp_fx(zn);
        meta = status | kStFrozen | ev;
        return kNoCell;
    }
    const Words u = rng_words(R, pid, step, 2u);
    // an ion neutralised at a wall comes back at T_refl; atoms and the gas
    // reinjected at the inlet at T0
    const float sig = Q >= 1 ? R.sig_refl : R.sig0;
    if (kind == 4) {
        X = R.inlet_X; Y = R.inlet_Y; Z = R.inlet_Z;
        emit(R.sig0, 0.f, 0.f, 1.f, 1.f, 0.f, 0.f, 0.f, 1.f, 0.f, u, vx, vy, vz);
    } else if (kind == 1) {
        const double rc = sqrt(cxd * cxd + cyd * cyd);
        const float ux = (float)(cxd / rc), uy = (float)(cyd / rc);
        const double sc = (R.R0_d - R.eps_wall_d) / rc;
        X = (int32_t)rint(cxd * sc / sxy);
        Y = (int32_t)rint(cyd * sc / sxy);
        Z = (int32_t)(long long)rint(czd / szd - 2147483648.0);
        emit(sig, -ux, -uy, 0.f, -uy, ux, 0.f, 0.f, 0.f, 1.f, u, vx, vy, vz);
    } else if (kind == 2) {
        X = (int32_t)rint(cxd / sxy);
        Y = (int32_t)rint(cyd / sxy);
        Z = (int32_t)(long long)rint(R.eps_wall_d / szd - 2147483648.0);
        emit(sig, 0.f, 0.f, 1.f, 1.f, 0.f, 0.f, 0.f, 1.f, 0.f, u, vx, vy, vz);
    } else {
        X = (int32_t)rint(cxd / sxy);
        Y = (int32_t)rint(cyd / sxy);
        Z = (int32_t)(long long)rint((R.L_d - R.eps_wall_d) / szd - 2147483648.0);
        emit(sig, 0.f, 0.f, -1.f, 1.f, 0.f, 0.f, 0.f, 1.f, 0.f, u, vx, vy, vz);
    }
    meta = status | ev;   // Q = 0: the particle comes back as an atom
    return ngp_cell(R, X, Y, Z);
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA engine) between global and shared memory, and
// the mbarrier that tracks the loads.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// bounded wait for phase `parity` of the barrier; false if the limit ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    const uint32_t a = smem_addr(bar);
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// global -> shared, `bytes` a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// shared -> global, same alignment rules
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// One stage of the tile pipeline: SoA copies of a tile's particles (kG
// float4 groups of four particles).
template <int kG>
struct Stage {
    int4 x[kG], y[kG], z[kG];
    float4 vx[kG], vy[kG], vz[kG];
    uint4 meta[kG];
    uint4 id[kG];
};

template <int kG, int kS>
struct StepShared {
    Stage<kG> st[kS];
    RunDev rs[kS];         // batch form: the stage's run parameter block (copied with the tile)
    uint32_t npart[kS];    // Coulomb participants of the stage's tile
    uint32_t lastk;        // the block's last tile loaded (counted from 0), ~0 before the first
    uint64_t bar[kS];
    int failed;
};

// Launch shape of the step kernel: kT threads per block, kV particles per
// thread and tile (tile = kT kV particles), kS pipeline stages in shared
// memory, and the resident blocks per SM asked of the register allocator:
// about 1280 threads per SM with two stages; with three, as many blocks as
// the stages' shared memory leaves room for.
template <int kT, int kV, int kS = 2>
struct Shape {
    static constexpr int threads = kT, vec = kV, stages = kS, tile = kT * kV, groups = kT * kV / 4;
    static constexpr int min_blocks =
        kS == 2 ? (kT == 128 ? 10 : (kT == 256 ? ECRIS_STEP_MIN_BLOCKS : 2))
                : (kT * kV <= 256 ? (kT == 128 ? 8 : 5) : 4);
};

__device__ __forceinline__ float& sf(float4* a, uint32_t i) { return reinterpret_cast<float*>(a)[i]; }
__device__ __forceinline__ uint32_t& su(uint4* a, uint32_t i) { return reinterpret_cast<uint32_t*>(a)[i]; }
__device__ __forceinline__ int32_t& si(int4* a, uint32_t i) { return reinterpret_cast<int32_t*>(a)[i]; }

// issue the eight bulk loads of tile t into stage st (thread 0 only); in the
// batch form also the run's parameter block into *rs, on the same barrier
template <int kG>
__device__ __forceinline__ void load_tile(const RunDev& R, Stage<kG>& st, uint64_t* bar, uint32_t t, RunDev* rs)
{
    const uint32_t g0 = t * kG;
    const uint32_t ng = min((uint32_t)kG, R.n4 - g0);
    const uint32_t bytes = ng * 16u;
    mbar_expect_tx(bar, 8u * bytes + (rs ? (uint32_t)sizeof(RunDev) : 0u));
    if (rs) bulk_load(rs, &R, (uint32_t)sizeof(RunDev), bar);
    bulk_load(st.x, reinterpret_cast<const int4*>(R.x) + g0, bytes, bar);
    bulk_load(st.y, reinterpret_cast<const int4*>(R.y) + g0, bytes, bar);
    bulk_load(st.z, reinterpret_cast<const int4*>(R.z) + g0, bytes, bar);
    bulk_load(st.vx, reinterpret_cast<const float4*>(R.vx) + g0, bytes, bar);
    bulk_load(st.vy, reinterpret_cast<const float4*>(R.vy) + g0, bytes, bar);
    bulk_load(st.vz, reinterpret_cast<const float4*>(R.vz) + g0, bytes, bar);
    bulk_load(st.meta, reinterpret_cast<const uint4*>(R.meta) + g0, bytes, bar);
    bulk_load(st.id, reinterpret_cast<const uint4*>(R.id) + g0, bytes, bar);
}

// NGP deposition of one particle per lane (the whole warp calls it), summed
// over runs of neighbouring lanes in the same cell (particles are kept sorted
// by cell, so neighbours mostly are): a segmented inclusive scan of the charge
// over each run's lanes (shuffles that stay inside the run), and the last lane
// of the run adds count << 32 | charge for it.
__device__ __forceinline__ void deposit_warp(const RunDev& R, uint32_t cell, uint32_t Q)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, cell, 1);
    const uint32_t heads = __ballot_sync(0xFFFFFFFFu, lane == 0 || prev != cell);
    const uint32_t h = 31u - (uint32_t)__clz(heads & (0xFFFFFFFFu >> (31u - lane)));   // first lane of the run
    uint32_t q = Q;
    if (__any_sync(0xFFFFFFFFu, Q != 0u)) {   // a warp of atoms deposits counts only
#pragma unroll
        for (uint32_t d = 1; d < 32u; d <<= 1) {
            const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, q, d);
            if (lane >= h + d) q += o;   // lane - d lies in the same run
        }
    }
    const bool last = lane == 31u || ((heads >> (lane + 1u)) & 1u);
    if (last && cell != kNoCell)
        atomicAdd(R.dep + cell, ((unsigned long long)(lane - h + 1u) << 32) | (unsigned long long)q);
}

// Publish this lane's Coulomb participant (ck != kNoCell) for the collision
// kernels: a slot in the tile's list (one shared-memory atomic per warp) and
// a count in its cell (one global reduction per run of neighbouring lanes in
// the same cell; the whole warp calls this)
__device__ __forceinline__ void publish_warp(const RunDev& R, uint32_t& npart, uint32_t t, uint32_t tile,
                                             uint32_t slot_in_run, uint32_t ck, uint32_t id, float vx, float vy,
                                             float vz, uint32_t Q)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t part = __ballot_sync(0xFFFFFFFFu, ck != kNoCell);
    if (!part) return;
    uint32_t base = 0;
    if (lane == (uint32_t)(__ffs(part) - 1)) base = atomicAdd(&npart, (uint32_t)__popc(part));
    base = __shfl_sync(0xFFFFFFFFu, base, __ffs(part) - 1);
    const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, ck, 1);
    const uint32_t heads = __ballot_sync(0xFFFFFFFFu, lane == 0 || prev != ck);
    if (ck == kNoCell) return;
    const uint32_t slot = t * tile + base + (uint32_t)__popc(part & ((1u << lane) - 1u));
    R.plist[slot] = make_uint4(slot_in_run, ck, id, 0u);
    R.pvel[slot] = make_float4(vx, vy, vz, __uint_as_float(Q));
    // every lane of a run shares ck, so all of them take part
    if (lane == 31 || ((heads >> (lane + 1)) & 1u)) {
        const uint32_t h = 31u - (uint32_t)__clz(heads & (0xFFFFFFFFu >> (31u - lane)));
        atomicAdd(R.ccount + ck, lane - h + 1u);
    }
}

// Where the tiles come from: one run (its parameter block a kernel argument)
// or a batch of runs (parameter blocks in device memory and a work list of
// (run, tile) items; the block stages the current item's block in shared
// memory).
struct SingleRun {
    const RunDev& R;
    uint32_t ntiles;
    __device__ __forceinline__ uint32_t count() const { return ntiles; }
    __device__ __forceinline__ uint2 item(uint32_t i) const { return make_uint2(0u, i); }
    __device__ __forceinline__ const RunDev& global(uint32_t) const { return R; }
};

struct BatchRuns {
    const RunDev* runs;
    const uint2* items;
    uint32_t nitems;
    __device__ __forceinline__ uint32_t count() const { return nitems; }
    __device__ __forceinline__ uint2 item(uint32_t i) const { return items[i]; }
    __device__ __forceinline__ const RunDev& global(uint32_t r) const { return runs[r]; }
};

// List the particles of this lane that left the chamber (leave) for the
// leaver pass: one global atomic per warp.
__device__ __forceinline__ void list_leavers(const RunDev& R, bool leave, uint32_t slot)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, leave);
    if (!m) return;
    uint32_t base = 0;
    if (lane == (uint32_t)(__ffs(m) - 1)) base = atomicAdd(R.nleave, (uint32_t)__popc(m));
    base = __shfl_sync(0xFFFFFFFFu, base, __ffs(m) - 1);
    if (leave) R.leave[base + (uint32_t)__popc(m & ((1u << lane) - 1u))] = slot;
}

// wait until at most n of this thread's bulk store groups have not yet read
// their shared memory
template <int n>
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(n) : "memory"); }

// Persistent pass over the work items with kS shared-memory stages: while the
// block advances one tile, the TMA engine brings in the next and the bulk
// stores of the previous ones drain.  As tile j starts, thread 0 loads tile
// j + 1 into stage (j + 1) mod kS, which tile j + 1 - kS used last: with two
// stages that is tile j - 1, whose stores (issued a moment before) must first
// have read the stage; with three it is tile j - 2, whose stores had a whole
// tile's time to do so.  The particles are kept sorted by (ion/atom, cell),
// so each thread takes slots tid, tid + kT, ... straight from the stage and
// the warps stay on one branch.
template <bool kBatch, bool kVar, class Sh, class Src>
__device__ __forceinline__ void step_tiles(StepShared<Sh::groups, Sh::stages>& S, const Src& src)
{
    constexpr uint32_t kT = Sh::threads, kV = Sh::vec, kTl = Sh::tile, kG = Sh::groups, kS = Sh::stages;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (uint32_t u = 0; u < kS; ++u) {
            mbar_init(&S.bar[u], 1);
            S.npart[u] = 0u;
        }
        S.failed = 0;
        S.lastk = ~0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const uint32_t nitems = src.count();
    uint32_t i = blockIdx.x;
    if (tid == 0 && i < nitems) {
        const uint2 it0 = src.item(i);
        S.lastk = 0u;
        load_tile(src.global(it0.x), S.st[0], &S.bar[0], it0.y, kBatch ? &S.rs[0] : nullptr);
    }
    // this tile's stage s and the parity ph of its barrier phase (with two
    // stages both follow from the tile count it)
    uint32_t s3 = 0, ph3 = 0;
    for (uint32_t it = 0; i < nitems; ++it, i += gridDim.x) {
        const uint32_t s = kS == 2 ? (it & 1u) : s3;
        const uint32_t ph = kS == 2 ? ((it >> 1) & 1u) : ph3;
        Stage<kG>& st = S.st[s];
        const uint2 item = src.item(i);
        const uint32_t in = i + gridDim.x;
        if (tid == 0 && in < nitems) {
            const uint32_t sn = s + 1u == kS ? 0u : s + 1u;
            const uint2 itn = src.item(in);
            bulk_wait_read<kS - 2>();   // the stores of the stage's last tile have read it
            S.lastk = it + 1u;
            load_tile(src.global(itn.x), S.st[sn], &S.bar[sn], itn.y, kBatch ? &S.rs[sn] : nullptr);
        }
        // a warp whose wait ran out (in any lane) leaves the tile alone; the
        // block learns of it at the barrier and stops there
        const bool ok = __all_sync(0xFFFFFFFFu, mbar_wait(&S.bar[s], ph));
        const uint32_t t = item.y;
        if (ok) {
            const RunDev& R = kBatch ? S.rs[s] : src.global(0);
            const bool coulomb = (R.flags & kFCoulomb) != 0;
            const uint32_t step = *R.step;
            const uint32_t nslot = min(kTl, 4u * (R.n4 - t * kG));
            // thread tid takes slots tid, tid + kT, ... (kV of them) of the
            // tile: a warp covers 32 consecutive slots (one kind of particle, few
            // cells), the shared-memory accesses are free of bank conflicts, and
            // every particle runs through the same single copy of the code
#pragma unroll 1
            for (uint32_t j = 0; j < kV; ++j) {
                const uint32_t k = (uint32_t)tid + j * kT;
                uint32_t meta = k < nslot ? su(st.meta, k) : kStPad;
                int32_t x = si(st.x, k), y = si(st.y, k), z = si(st.z, k);
                float vx = sf(st.vx, k), vy = sf(st.vy, k), vz = sf(st.vz, k);
                const uint32_t id = su(st.id, k);
                uint32_t ck, dc;
                const bool leave = step_particle<kVar>(R, id, step, x, y, z, vx, vy, vz, meta, ck, dc);
                deposit_warp(R, dc, meta & kQMask);
                list_leavers(R, leave, t * kTl + k);
                if (k < nslot) {
                    si(st.x, k) = x; si(st.y, k) = y; si(st.z, k) = z;
                    sf(st.vx, k) = vx; sf(st.vy, k) = vy; sf(st.vz, k) = vz;
                    su(st.meta, k) = meta;
                }
                if (coulomb) publish_warp(R, S.npart[s], t, kTl, t * kTl + k, ck, id, vx, vy, vz, meta & kQMask);
            }
        }
        fence_proxy_async();    // make this thread's stage writes visible to the bulk stores
        // One block barrier per tile, before the stores: every thread has
        // written its slots, and none reads the stage again before it is
        // reloaded.  A stage's participant count is reset here and used
        // again kS tiles on, past the next barrier.
        if (__syncthreads_or(ok ? 0 : 1)) {
            if (tid == 0) {
                S.failed = 1;
                atomicExch(src.global(item.x).err, kErrTimeout);
            }
            break;
        }
        if (tid == 0) {
            const RunDev& R = kBatch ? S.rs[s] : src.global(0);
            const bool coulomb = (R.flags & kFCoulomb) != 0;
            const uint32_t g0 = t * kG;
            const uint32_t bytes = min(kG, R.n4 - g0) * 16u;
            bulk_store(reinterpret_cast<int4*>(R.x) + g0, st.x, bytes);
            bulk_store(reinterpret_cast<int4*>(R.y) + g0, st.y, bytes);
            bulk_store(reinterpret_cast<int4*>(R.z) + g0, st.z, bytes);
            bulk_store(reinterpret_cast<float4*>(R.vx) + g0, st.vx, bytes);
            bulk_store(reinterpret_cast<float4*>(R.vy) + g0, st.vy, bytes);
            bulk_store(reinterpret_cast<float4*>(R.vz) + g0, st.vz, bytes);
            bulk_store(reinterpret_cast<uint4*>(R.meta) + g0, st.meta, bytes);
            bulk_commit();
            if (coulomb) R.tcount[t] = S.npart[s];
            S.npart[s] = 0u;
        }
        if (kS != 2 && ++s3 == kS) {
            s3 = 0u;
            ph3 ^= 1u;
        }
    }
    pdl_trigger();              // the leaver pass may be scheduled (it waits for this grid)
    if (tid == 0) {
        bulk_wait_all();        // stores complete before the block retires
        if (S.failed) {
            // loads issued into a stage may still land: the block's tile k
            // went into stage k mod kS at phase k / kS; wait (bounded) for
            // each stage's last one (phases complete in order)
            const uint32_t last = S.lastk;
            for (uint32_t u = 0; u < kS && u <= last && last != ~0u; ++u) {
                const uint32_t k = last - (last - u) % kS;
                mbar_wait(&S.bar[u], (k / kS) & 1u);
            }
        }
    }
}

using DefaultShape = Shape<kThreads, kVec>;

template <bool kVar>
__global__ void __launch_bounds__(kThreads, kStepMinBlocks) k_step(const __grid_constant__ RunDev R, uint32_t ntiles)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    auto& S = *reinterpret_cast<StepShared<DefaultShape::groups, DefaultShape::stages>*>(smem_raw);
    step_tiles<false, kVar, DefaultShape>(S, SingleRun{R, ntiles});
}

// batch form: one persistent launch over the tiles of many runs, in one of
// the launch shapes the batch autotuner chooses from
template <bool kVar, class Sh>
__global__ void __launch_bounds__(Sh::threads, Sh::min_blocks) k_step_batch(const RunDev* __restrict__ runs,
                                                                            const uint2* __restrict__ items,
                                                                            uint32_t nitems)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    auto& S = *reinterpret_cast<StepShared<Sh::groups, Sh::stages>*>(smem_raw);
    step_tiles<true, kVar, Sh>(S, BatchRuns{runs, items, nitems});
}

// The leaver pass of one run: finish the step of every listed particle, add
// its deposit, and clear the list.  Threads [tid0, tid0 + nthr) of the grid
// share the work.
__device__ __forceinline__ void leave_run(const RunDev& R, uint32_t n, uint32_t tid0, uint32_t nthr)
{
    const uint32_t step = *R.step;
    for (uint32_t e = tid0; e < n; e += nthr) {
        const uint32_t i = R.leave[e];
        int32_t X = R.x[i], Y = R.y[i], Z = R.z[i];
        float vx = R.vx[i], vy = R.vy[i], vz = R.vz[i];
        uint32_t meta = R.meta[i];
        const uint32_t cell = leave_particle(R, R.id[i], step, X, Y, Z, vx, vy, vz, meta);
        if (cell != kNoCell) atomicAdd(R.dep + cell, 1ull << 32);   // Q = 0: count only
        R.x[i] = X;
        R.y[i] = Y;
        R.z[i] = Z;
        R.vx[i] = vx;
        R.vy[i] = vy;
        R.vz[i] = vz;
        R.meta[i] = meta;
    }
}

// last block of a grid (after every block's work is visible): ticket reset
__device__ __forceinline__ bool last_block(unsigned int* ticket)
{
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1 ? 1 : 0;
        if (last) *ticket = 0u;
    }
    __syncthreads();
    return last != 0;
}

// one run; the last block clears the list and, with bump_step, advances the
// run's step counter (runs with Coulomb collisions advance it in the
// collision kernels)
__global__ void __launch_bounds__(256) k_leave(const __grid_constant__ RunDev R, unsigned int* ticket, int bump_step)
{
    pdl_wait();
    pdl_trigger();
    const uint32_t n = *R.nleave;
    leave_run(R, n, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
    if (last_block(ticket) && threadIdx.x == 0) {
        *R.nleave = 0u;
        if (bump_step) *R.step += 1u;
    }
}

// every run of a batch: block b takes runs b, b + grid, ...; the last block
// clears the lists and advances the step counter of every run without
// Coulomb collisions (nothing reads those counters again in this step; the
// collision kernels of the other runs advance their own)
__global__ void __launch_bounds__(256) k_leave_batch(const RunDev* __restrict__ runs, uint32_t nruns,
                                                     unsigned int* ticket)
{
    pdl_wait();
    for (uint32_t r = blockIdx.x; r < nruns; r += gridDim.x) {
        const RunDev& R = runs[r];
        if (!R.step) continue;
        leave_run(R, *R.nleave, threadIdx.x, blockDim.x);
    }
    if (last_block(ticket))
        for (uint32_t r = threadIdx.x; r < nruns; r += blockDim.x)
            if (runs[r].step) {
                *runs[r].nleave = 0u;
                if (!(runs[r].flags & kFCoulomb)) *runs[r].step += 1u;
            }
}

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

// range b of the collision kernel (stride participants a range) starts at the
// first cell c with coff[c] >= b stride: cell c starts the ranges b with
// coff[c - 1] < b stride <= coff[c], and each of them records coff[c], its
// first participant
__device__ __forceinline__ void mark_ranges(const RunDev& R, uint32_t c, uint32_t prev, uint32_t cur,
                                            uint32_t stride)
{
    const uint32_t b0 = c == 0 ? 0u : prev / stride + 1u;
    for (uint32_t b = b0; b <= cur / stride; ++b) R.cstart[b] = cur;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// One-pass exclusive scan of ccount into coff (coff[ncells] = total) with
// decoupled look-back: each block takes the next scan tile in ticket order,
// scans its kScanBlock counts, publishes the tile's total, then adds up the
// totals (or the first inclusive prefix) of the tiles before it.  A status
// word is epoch << 33 | inclusive << 32 | value; the epoch (launch number,
// from the ticket) tells this launch's words from stale ones.  A wait that
// runs out of its bounded spin sets the run's error word.  The kernel also
// marks where the collision kernel's ranges start.
//
// It is the first kernel after the step kernel in a one-run step with
// Coulomb collisions, and blocks past the nscan scan tiles do that step's
// leaver pass meanwhile if do_leave (the leavers take no part in the
// collisions); the collision kernel clears the leaver list at its end.
// ntile = blocks in all; it must not change between the launches of a run
// (the tickets' cycle gives the epoch), so a one-run step whose leaver pass
// ran on its own still launches the extra blocks, with do_leave = 0.
__global__ void __launch_bounds__(kScanThreads) k_scan(const __grid_constant__ RunDev R, uint32_t ncells,
                                                      uint32_t ntile, uint32_t nscan, int do_leave)
{
    __shared__ uint32_t wsum[kScanThreads / 32], wred[kScanThreads / 32];
    __shared__ uint32_t s_tile, s_epoch, s_agg, s_first, s_bad, s_stride, s_max;
    pdl_wait();
    pdl_trigger();   // the scatter's blocks may be scheduled; they wait for this grid
    if (threadIdx.x == 0) {
        s_stride = R.crange[0];
        s_max = 0u;
        const unsigned long long t = atomicAdd(R.cctr, 1ull);
        s_tile = (uint32_t)(t % ntile);
        s_epoch = (uint32_t)(t / ntile) + 1u;
    }
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= nscan) {   // the last tickets: the leaver pass
        if (do_leave)
            leave_run(R, *R.nleave, (tile - nscan) * blockDim.x + threadIdx.x, (ntile - nscan) * blockDim.x);
        return;
    }
    const unsigned long long ep = (unsigned long long)s_epoch << 33;
    const uint32_t base = tile * kScanBlock + threadIdx.x * kScanPerThread;
    uint32_t v[kScanPerThread];
    uint32_t sum = 0;
    // four counts per load where the group lies inside the mesh
#pragma unroll
    for (int j = 0; j < kScanPerThread; j += 4) {
        const uint32_t idx = base + j;
        if (idx + 3u < ncells) {
            const uint4 c4 = *reinterpret_cast<const uint4*>(R.ccount + idx);
            v[j] = c4.x; v[j + 1] = c4.y; v[j + 2] = c4.z; v[j + 3] = c4.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) v[j + k] = idx + k < ncells ? R.ccount[idx + k] : 0u;
        }
    }
    // the count of the cell before this thread's first (for its range marks)
    const uint32_t vprev = base > 0u && base - 1u < ncells ? R.ccount[base - 1u] : 0u;
    uint32_t vmax = 0;
#pragma unroll
    for (int j = 0; j < kScanPerThread; ++j) {
        sum += v[j];
        vmax = max(vmax, v[j]);
    }
    // the largest cell count, for the next step's range size
    vmax = __reduce_max_sync(0xFFFFFFFFu, vmax);
    if ((threadIdx.x & 31) == 0 && vmax) atomicMax(&s_max, vmax);
    const uint32_t stride = s_stride;
    const uint32_t incl = warp_incl_scan(sum);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0 && s_max) atomicMax(R.crange + 1, s_max);
    if (warp == 0) {
        const uint32_t w = lane < kScanThreads / 32 ? wsum[lane] : 0u;
        const uint32_t wi = warp_incl_scan(w);
        if (lane < kScanThreads / 32) wsum[lane] = wi - w;
        // the tile's total: publish it (tile 0 as its inclusive prefix)
        const uint32_t agg = __shfl_sync(0xFFFFFFFFu, wi, kScanThreads / 32 - 1);
        if (lane == 0) {
            st_release(R.cstat + tile, ep | (tile == 0 ? (1ull << 32) : 0ull) | agg);
            s_agg = agg;
            s_first = kScanThreads;
            s_bad = 0u;
        }
    }
    __syncthreads();
    // look back over up to kScanThreads earlier tiles a round, thread k reading
    // tile p - k, and add up the totals down to the nearest inclusive prefix:
    // every tile's total is published before its look-back starts, so one
    // round reaches tile 0 when there are at most kScanThreads tiles
    uint32_t prefix = 0;
    if (tile > 0) {
        for (int p = (int)tile - 1; p >= 0; p -= kScanThreads) {
            const int q = p - (int)threadIdx.x;
            unsigned long long st = 0;
            if (q >= 0) {
                uint32_t it = 0;
                do {
                    st = ld_acquire(R.cstat + q);
                } while ((st >> 33) != (ep >> 33) && ++it < kWaitLimit);
                if ((st >> 33) != (ep >> 33)) s_bad = 1u;
                if (st & (1ull << 32)) atomicMin(&s_first, threadIdx.x);
            }
            __syncthreads();
            const uint32_t first = s_first;
            const uint32_t val = __reduce_add_sync(0xFFFFFFFFu, (q >= 0 && threadIdx.x <= first) ? (uint32_t)st : 0u);
            if (lane == 0) wred[warp] = val;
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kScanThreads / 32; ++k) prefix += wred[k];
            if (first < (uint32_t)kScanThreads) break;
            __syncthreads();   // every thread has read wred before the next round writes it
        }
        if (threadIdx.x == 0) {
            if (s_bad) atomicExch(R.err, kErrTimeout);
            st_release(R.cstat + tile, ep | (1ull << 32) | (prefix + s_agg));
        }
    }
    uint32_t o[kScanPerThread];
    uint32_t cur = prefix + wsum[warp] + incl - sum;
#pragma unroll
    for (int j = 0; j < kScanPerThread; ++j) {
        o[j] = cur;
        cur += v[j];
    }
    if (base + kScanPerThread <= ncells) {
#pragma unroll
        for (int j = 0; j < kScanPerThread; j += 4)
            *reinterpret_cast<uint4*>(R.coff + base + j) = make_uint4(o[j], o[j + 1], o[j + 2], o[j + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < kScanPerThread; ++j)
            if (base + j < ncells) R.coff[base + j] = o[j];
    }
    // the collision kernel's ranges that start at each cell
#pragma unroll
    for (int j = 0; j < kScanPerThread; ++j) {
        const uint32_t idx = base + j;
        if (idx < ncells) {
            mark_ranges(R, idx, j > 0 ? o[j - 1] : o[0] - vprev, o[j], stride);
            if (idx == ncells - 1) {
                R.coff[ncells] = o[j] + v[j];
                mark_ranges(R, ncells, o[j], o[j] + v[j], stride);
            }
        }
    }
}


// Fold the packed per-step deposit into the time-summed count and charge
// grids and clear it.
__global__ void k_fold(const __grid_constant__ RunDev R, uint32_t ncells,
                       unsigned long long* __restrict__ count, unsigned long long* __restrict__ charge)
{
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
        const unsigned long long v = R.dep[c];
        if (v) {
            count[c] += v >> 32;
            charge[c] += v & 0xFFFFFFFFull;
            R.dep[c] = 0ull;
        }
    }
}

// Number of particles in the chamber per charge state.
__global__ void k_census(const __grid_constant__ RunDev R, uint32_t n4,
                         unsigned long long* __restrict__ census)
{
    __shared__ unsigned int h[kQSlots];
    for (int i = threadIdx.x; i < kQSlots; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n4; g += gridDim.x * blockDim.x) {
        const uint4 m = reinterpret_cast<const uint4*>(R.meta)[g];
        const uint32_t mm[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (!(mm[j] & (kStFrozen | kStPad))) atomicAdd(&h[mm[j] & kQMask], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kQSlots; i += blockDim.x)
        if (h[i]) atomicAdd(census + i, (unsigned long long)h[i]);
}

struct SoaPtrs { float* p[6]; };

// v * (hi + lo) rounded to the nearest integer: the FP32 product p = v hi is
// an integer once |p| >= 2^24, and its rounding error (exact by FMA) plus
// v lo is added as a small correction.  Float-to-64-bit conversions run on
// the narrow FP64 pipe, so values inside the signed or unsigned 32-bit range
// (every position but the chamber's outermost points) convert in 32 bits, to
// the same integers
__device__ __forceinline__ long long scale_round(float v, float hi, float lo)
{
    const float p = v * hi;
    const float e = fmaf(v, hi, -p) + v * lo;
    const float r = rintf(p);
    long long P;
    if (fabsf(r) < 2147483648.0f) P = (long long)__float2int_rn(r);
    else if (r >= 0.0f && r < 4294967296.0f) P = (long long)__float2uint_rn(r);
    else P = (long long)r;
    return P + (long long)__float2int_rn(e + (p - r));
}

// metres -> fixed point, rounded to nearest, saturated
__device__ __forceinline__ void store_fx(SoaPtrs soa, uint32_t i, float x, float y, float z, const LoadCheck& lc)
{
    const long long lim = 2147483647ll;
    const long long X = max(min(scale_round(x, lc.inv_sxy_hi, lc.inv_sxy_lo), lim), -lim - 1);
    const long long Y = max(min(scale_round(y, lc.inv_sxy_hi, lc.inv_sxy_lo), lim), -lim - 1);
    const long long Z = max(min(scale_round(z, lc.inv_sz_hi, lc.inv_sz_lo) - 2147483648ll, lim), -lim - 1);
    reinterpret_cast<int32_t*>(soa.p[0])[i] = (int32_t)X;
    reinterpret_cast<int32_t*>(soa.p[1])[i] = (int32_t)Y;
    reinterpret_cast<int32_t*>(soa.p[2])[i] = (int32_t)Z;
}

__global__ void k_load_init(LoadCheck lc, SoaPtrs soa, const uint8_t* __restrict__ q8,
                            uint32_t* __restrict__ meta, uint32_t* __restrict__ id, uint32_t n, uint32_t cap,
                            unsigned int* __restrict__ bad)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
        id[i] = i;
        if (i < n) {
            const float x = soa.p[0][i], y = soa.p[1][i], z = soa.p[2][i];
            const float vx = soa.p[3][i], vy = soa.p[4][i], vz = soa.p[5][i];
            const uint32_t q = q8[i];
            const bool ok = (x * x + y * y <= lc.R0sq) && (z >= 0.0f) && (z <= lc.L) &&
                            isfinite(vx) && isfinite(vy) && isfinite(vz) && q <= lc.qmax;
            if (!ok) {
                atomicAdd(bad, 1u);
                atomicMin(bad + 1, i);
            }
            meta[i] = q;
            store_fx(soa, i, x, y, z, lc);
        } else {
            store_fx(soa, i, lc.inlet_x, lc.inlet_y, lc.inlet_z, lc);
            soa.p[3][i] = 0.0f;
            soa.p[4][i] = 0.0f;
            soa.p[5][i] = 0.0f;
            meta[i] = kStPad;
        }
    }
}

}  // namespace

cudaError_t launch_load_init(const LoadCheck& lc, float* const soa[6], const uint8_t* q8, uint32_t* meta,
                             uint32_t* id, uint32_t n, uint32_t cap, unsigned int* bad, cudaStream_t s)
{
    SoaPtrs p;
    for (int k = 0; k < 6; ++k) p.p[k] = soa[k];
    const int threads = 256;
    int blocks = (int)((cap + threads - 1) / threads);
    if (blocks > 8192) blocks = 8192;
    k_load_init<<<blocks, threads, 0, s>>>(lc, p, q8, meta, id, n, cap, bad);
    return cudaGetLastError();
}

int step_blocks_per_sm()
{
    const int smem = (int)sizeof(StepShared<DefaultShape::groups, DefaultShape::stages>);
    if (cudaFuncSetAttribute(k_step<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_step<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return 1;
    int b = 0, bv = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step<false>, kThreads, smem) != cudaSuccess || b < 1) b = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bv, k_step<true>, kThreads, smem) != cudaSuccess || bv < 1)
        bv = 1;
    return b < bv ? b : bv;
}

// the batch kernel of launch shape Sh: resident blocks per SM (the smaller
// of its two instantiations), and the launch
template <class Sh>
int batch_bps()
{
    constexpr int smem = (int)sizeof(StepShared<Sh::groups, Sh::stages>);
    if (cudaFuncSetAttribute(k_step_batch<false, Sh>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_step_batch<true, Sh>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess)
        return 1;
    int b = 0, bv = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step_batch<false, Sh>, Sh::threads, smem) !=
            cudaSuccess ||
        b < 1)
        b = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bv, k_step_batch<true, Sh>, Sh::threads, smem) !=
            cudaSuccess ||
        bv < 1)
        bv = 1;
    return b < bv ? b : bv;
}

template <class Sh>
void batch_launch_shape(const RunDev* runs, const uint2* items, uint32_t nitems, int grid, bool variants,
                        cudaStream_t s)
{
    constexpr size_t smem = sizeof(StepShared<Sh::groups, Sh::stages>);
    if (variants) k_step_batch<true, Sh><<<grid, Sh::threads, smem, s>>>(runs, items, nitems);
    else k_step_batch<false, Sh><<<grid, Sh::threads, smem, s>>>(runs, items, nitems);
}

// apply F to the Shape type of launch shape k (kStepShapes of them)
template <class F>
auto with_shape(int k, F f)
{
    switch (k) {
    case 0: return f(Shape<128, 1>{});
    case 1: return f(Shape<128, 2>{});
    case 2: return f(Shape<128, 4>{});
    case 3: return f(Shape<256, 1>{});
    case 5: return f(Shape<256, 4>{});
    case 6: return f(Shape<512, 1>{});
    case 7: return f(Shape<512, 2>{});
    case 8: return f(Shape<512, 4>{});
    case 9: return f(Shape<128, 2, 3>{});
    case 10: return f(Shape<256, 1, 3>{});
    case 11: return f(Shape<256, 2, 3>{});
    default: return f(Shape<256, 2>{});
    }
}

int step_batch_blocks_per_sm(int shape)
{
    return with_shape(shape, [](auto sh) { return batch_bps<decltype(sh)>(); });
}

cudaError_t launch_step_batch(const RunDev* runs, const uint2* items, uint32_t nitems, int grid, bool variants,
                              int shape, cudaStream_t s)
{
    if (nitems > 0) {
        if (grid > (int)nitems) grid = (int)nitems;
        with_shape(shape, [&](auto sh) {
            batch_launch_shape<decltype(sh)>(runs, items, nitems, grid, variants, s);
            return 0;
        });
    }
    return cudaGetLastError();
}

cudaError_t launch_step(const RunDev& R, uint32_t ntiles, int grid, cudaStream_t s)
{
    if (ntiles == 0) return cudaSuccess;
    if (grid > (int)ntiles) grid = (int)ntiles;
    constexpr size_t smem = sizeof(StepShared<DefaultShape::groups, DefaultShape::stages>);
    if ((R.flags & kFVariants) || R.btab) k_step<true><<<grid, kThreads, smem, s>>>(R, ntiles);
    else k_step<false><<<grid, kThreads, smem, s>>>(R, ntiles);
    return cudaGetLastError();
}

cudaError_t launch_scan(const RunDev& R, uint32_t ncells, uint32_t nscan, uint32_t leave_blocks, int do_leave,
                        cudaStream_t s)
{
    return launch_pdl(k_scan, dim3(nscan + leave_blocks), dim3(kScanThreads), 0, s, R, ncells, nscan + leave_blocks,
                      nscan, do_leave);
}

cudaError_t launch_leave(const RunDev& R, unsigned int* ticket, int bump_step, cudaStream_t s)
{
    return launch_pdl(k_leave, dim3(kLeaveBlocks), dim3(256), 0, s, R, ticket, bump_step);
}

cudaError_t launch_leave_batch(const RunDev* runs, uint32_t nruns, unsigned int* ticket, cudaStream_t s)
{
    if (nruns == 0) return cudaSuccess;
    return launch_pdl(k_leave_batch, dim3(nruns < (uint32_t)kLeaveBlocks ? nruns : (uint32_t)kLeaveBlocks),
                      dim3(256), 0, s, runs, nruns, ticket);
}

cudaError_t launch_fold(const RunDev& R, uint32_t ncells, unsigned long long* count, unsigned long long* charge,
                        cudaStream_t s)
{
    const int threads = 256;
    int blocks = (int)((ncells + threads - 1) / threads);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_fold<<<blocks, threads, 0, s>>>(R, ncells, count, charge);
    return cudaGetLastError();
}

cudaError_t launch_census(const RunDev& R, uint32_t n4, unsigned long long* census, cudaStream_t s)
{
    const int threads = 256;
    int blocks = (int)((n4 + threads - 1) / threads);
    if (blocks > 2048) blocks = 2048;
    if (blocks < 1) blocks = 1;
    k_census<<<blocks, threads, 0, s>>>(R, n4, census);
    return cudaGetLastError();
}

}  // namespace ecris
