// Served form of the ECRIS ion time step: a request loop that keeps one batch
// of runs resident on the device and admits queued runs as slots and memory
// free up (continuous batching).
//
// The loop, on its own thread, per tick:
//   1. admit queued requests in arrival order while the batch's memory
//      budget and the slot limit allow (a request that does not fit waits, and
//      the ones behind it wait too, so arrival order is kept); a new run is
//      set up on its own stream while the batch's queued steps run;
//   2. enqueue steps_per_tick steps of the batch (one graph replay per step)
//      and, for every run whose own step count reaches a multiple of its
//      window, a copy of its tallies into pinned memory (a snapshot);
//   3. while those steps run, read the snapshots of the previous tick and
//      apply the convergence rule (stationary extracted currents, Sec. II) or
//      the step cap; retire finished runs, which frees their memory for the
//      queue in stream order.
// A run retired at a boundary has run one tick past it; its result is the
// snapshot at the boundary.  Because the rule only looks at a run's own
// counters at its own window boundaries, and a run in a batch evolves exactly
// as it does alone, the result of a request does not depend on what else is
// being served.
//
// Calibration jobs ride on the same loop: a job is a sequence of requests of
// one base run with the weight and warm-electron temperature it adjusts; when
// one of its runs retires, the loop records the run's last-window flow and
// power and queues the next run, until both meet their targets.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ecris.h"
#include "ecris_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// a request with every pointer replaced by owned copies
struct OwnedRequest {
    ecris_request r;
    std::vector<float> E, ne_cells, xyzv[6];
    std::vector<double> ip, axial;
    std::vector<int32_t> nout;
    std::vector<uint8_t> q;
};

struct CalibJob;

struct Served {
    int64_t ticket = 0;
    CalibJob* job = nullptr;         // the calibration job this run belongs to, if any
    std::unique_ptr<OwnedRequest> req;
    ecris_result res;
    int32_t run = -1;
    std::vector<int64_t> last_ext;   // extracted counts at the previous window boundary
    std::vector<double> last_cur;    // currents of the previous window
    std::vector<int64_t> last_dn;    // extractions by Q in the previous window
    double last_energy_J = 0.0;      // energy carried out up to the previous window boundary
    bool have_prev = false;
    uint64_t issued = 0;             // steps enqueued for the run
    uint64_t snap_steps = 0;         // steps at its latest snapshot
    bool ne_failed = false;          // a self-consistent n_e update could not be enqueued
    ecris::TallySnapshot* snap = nullptr;   // pinned
    cudaEvent_t ev = nullptr;        // the snapshot has landed
};

// a calibration job: its base request (owned), targets and history
struct CalibJob {
    int64_t id = 0;
    std::unique_ptr<OwnedRequest> base;
    double flow_target = 0.0, power_target = 0.0, tol = 0.0;
    int32_t max_iter = 1;
    double w = 0.0, Te = 0.0;        // inputs of the run in flight
    ecris_calib_result res;
};

}  // namespace

struct ecris_server {
    int device = 0;
    ecris_batch* batch = nullptr;
    size_t budget = 0;
    uint32_t steps_per_tick = 1;
    uint32_t max_active = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    std::string err;
    std::deque<Served*> queue;
    std::vector<Served*> active;
    std::map<int64_t, std::unique_ptr<Served>> all;
    std::map<int64_t, std::unique_ptr<CalibJob>> calibs;
    int64_t next_ticket = 1;
    int64_t next_job = 1;
    int64_t n_done = 0;
    double ion_steps = 0.0;
    double resident = 0.0;          // particles of the runs in the batch (loop thread)
    double tuned_at = 0.0;          // ... when the launch shape was last tuned
    int64_t n_tunes = 0;
    std::thread loop;
    // recycled pinned snapshot slots and events (only the loop thread uses them)
    std::vector<ecris::TallySnapshot*> free_snaps;
    std::vector<cudaEvent_t> free_events;
};

namespace {

double now_s(const ecris_server* s)
{
    return std::chrono::duration<double>(Clock::now() - s->t0).count();
}

void finish(ecris_server* s, Served* v, int32_t state, const char* msg)
{
    v->res.state = state;
    v->res.t_done = now_s(s);
    if (msg) std::strncpy(v->res.error, msg, sizeof v->res.error - 1);
}

// a pinned snapshot slot and an event for a newly admitted run
bool take_slot(ecris_server* s, Served* v)
{
    if (s->free_snaps.empty()) {
        ecris::TallySnapshot* p = nullptr;
        if (cudaMallocHost((void**)&p, sizeof(ecris::TallySnapshot)) != cudaSuccess) return false;
        s->free_snaps.push_back(p);
    }
    if (s->free_events.empty()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return false;
        s->free_events.push_back(e);
    }
    v->snap = s->free_snaps.back();
    s->free_snaps.pop_back();
    v->ev = s->free_events.back();
    s->free_events.pop_back();
    return true;
}

void give_slot(ecris_server* s, Served* v)
{
    if (v->snap) s->free_snaps.push_back(v->snap);
    if (v->ev) s->free_events.push_back(v->ev);
    v->snap = nullptr;
    v->ev = nullptr;
}

// the run's result at its latest snapshot (landed) into res; false on a
// device error
bool read_snapshot(ecris_server* s, Served* v, std::vector<int64_t>& ext, ecris_result& res)
{
    const int q1 = v->req->r.sp.qmax + 1;
    ext.assign(q1, 0);
    std::vector<int64_t> lost(q1, 0);
    if (v->snap->err) return false;
    ecris_diag_out d;
    std::memset(&d, 0, sizeof d);
    d.extracted = ext.data();
    d.lost = lost.data();
    ecris::batch_snapshot_diag(s->batch, v->run, *v->snap, v->snap_steps, &d);
    res.steps = d.steps;
    res.qmax = d.qmax;
    res.power_W = d.power_W;
    res.ke_lost_eV = d.ke_lost_eV;
    for (int q = 0; q < q1 && q < 64; ++q) {
        res.extracted[q] = ext[q];
        res.lost[q] = lost[q];
    }
    return true;
}

// the convergence rule at a window boundary (currents into res)
bool converged(Served* v, const std::vector<int64_t>& ext, ecris_result& res)
{
    const ecris_request& r = v->req->r;
    const int q1 = r.sp.qmax + 1;
    std::vector<double> cur(q1, 0.0);
    std::vector<int64_t> dn(q1, 0);
    int64_t events = 0;
    const double window_s = r.window_steps * r.dt;
    const double per_charge = 1.602176634e-19 * r.weight / window_s;   // current of one extracted charge
    for (int q = 0; q < q1; ++q) {
        dn[q] = ext[q] - (v->last_ext.empty() ? 0 : v->last_ext[q]);
        events += dn[q];
        cur[q] = q * per_charge * (double)dn[q];
    }
    for (int q = 0; q < q1 && q < 64; ++q) res.current_A[q] = cur[q];
    // gas flow and power losses over the window (the power from the
    // cumulative energy carried out, power_W times the run's time)
    res.flow_per_s = r.weight * (double)events / window_s;
    const double energy = res.power_W * (double)res.steps * r.dt;
    res.power_window_W = (energy - v->last_energy_J) / window_s;
    v->last_energy_J = energy;
    bool ok = false;
    if (v->have_prev && events >= r.min_events) {
        // two windows agree when their currents differ by at most rel_tol times
        // the larger, or by no more than the counting noise of the two windows
        // allows (three standard deviations of the difference of their
        // Poisson counts): the source is stationary when no drift shows above
        // what the extraction counts can resolve.  Two zero currents agree.
        auto agree = [&](double a, double b, double var_counts) {
            const double noise = 3.0 * per_charge * std::sqrt(var_counts);
            return std::abs(a - b) <= std::max(r.rel_tol * std::max(std::abs(a), std::abs(b)), noise);
        };
        double tot = 0.0, tot_prev = 0.0, var_tot = 0.0;
        for (int q = 0; q < q1; ++q) {
            tot += cur[q];
            tot_prev += v->last_cur[q];
            var_tot += (double)q * q * (double)(dn[q] + v->last_dn[q]);
        }
        ok = agree(tot, tot_prev, var_tot);
        std::vector<int> order(q1);
        for (int q = 0; q < q1; ++q) order[q] = q;
        std::sort(order.begin(), order.end(), [&](int a, int b) { return cur[a] > cur[b]; });
        for (int k = 0; k < 3 && k < q1 && ok; ++k) {
            const int q = order[k];
            ok = agree(cur[q], v->last_cur[q], (double)q * q * (double)(dn[q] + v->last_dn[q]));
        }
    }
    v->last_ext = ext;
    v->last_cur = cur;
    v->last_dn = dn;
    v->have_prev = true;
    return ok;
}

// a run of a calibration job: the base request with weight w and warm
// electron temperature Te, pointing into the job's owned arrays
std::unique_ptr<Served> calib_run(ecris_server* s, CalibJob* j)
{
    auto v = std::make_unique<Served>();
    auto o = std::make_unique<OwnedRequest>();
    o->r = j->base->r;
    o->r.weight = j->w;
    o->r.grid.Te_warm_eV = j->Te;
    v->req = std::move(o);
    v->job = j;
    std::memset(&v->res, 0, sizeof v->res);
    v->res.state = ECRIS_REQ_QUEUED;
    v->ticket = s->next_ticket++;
    v->res.t_submit = now_s(s);
    return v;
}

// a calibration run retired (s->mu held): record it and queue the next one,
// or finish the job
void calib_advance(ecris_server* s, Served* v, bool ok)
{
    CalibJob* j = v->job;
    ecris_calib_result& jr = j->res;
    if (!ok) {
        jr.state = ECRIS_REQ_FAILED;
        std::strncpy(jr.error, v->res.error, sizeof jr.error - 1);
        return;
    }
    const int k = jr.iterations;
    jr.weight[k] = j->w;
    jr.Te_warm_eV[k] = j->Te;
    jr.flow_per_s[k] = v->res.flow_per_s;
    jr.power_W[k] = v->res.power_window_W;
    jr.steps[k] = v->res.steps;
    jr.iterations = k + 1;
    const double F = v->res.flow_per_s, P = v->res.power_window_W;
    const bool met = F > 0.0 && P > 0.0 && std::abs(F / j->flow_target - 1.0) <= j->tol &&
                     std::abs(P / j->power_target - 1.0) <= j->tol;
    if (met || jr.iterations >= j->max_iter) {
        jr.met = met ? 1 : 0;
        jr.state = ECRIS_REQ_DONE;
        return;
    }
    // next inputs: flow and power scale with w; T_ew sets the energy per
    // particle carried out; each moves by at most a factor of 4
    auto clamp4 = [](double f) { return f < 0.25 ? 0.25 : (f > 4.0 ? 4.0 : f); };
    if (F > 0.0 && P > 0.0) {
        j->w *= clamp4(j->flow_target / F);
        j->Te *= clamp4((j->power_target / j->flow_target) / (P / F));
    } else {
        j->w *= 4.0;   // nothing left through the aperture in the window: more particles
    }
    auto n = calib_run(s, j);
    Served* raw = n.get();
    s->all[raw->ticket] = std::move(n);
    s->queue.push_back(raw);
    s->cv.notify_one();
}

void serve_loop(ecris_server* s)
{
    cudaSetDevice(s->device);
    const cudaStream_t bs = ecris::batch_stream(s->batch);
    std::vector<int64_t> ext;
    std::vector<Served*> waiting;   // runs with a snapshot enqueued in the previous tick
    for (;;) {
        // 1. admission, in arrival order
        std::vector<Served*> admit;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            if (s->stop) break;
            if (s->active.empty() && s->queue.empty() && waiting.empty()) {
                s->cv.wait_for(lock, std::chrono::milliseconds(20));
                continue;
            }
            size_t used = 0, budget = 0;
            ecris_batch_memory(s->batch, &used, &budget);
            while (!s->queue.empty()) {
                Served* v = s->queue.front();
                const ecris_request& r = v->req->r;
                const size_t need = ecris_run_bytes(r.n, r.grid.nx, r.grid.ny, r.grid.nz, (r.mcc.flags & ECRIS_F_COULOMB) != 0);
                if (budget && used + need > budget) break;
                if (s->max_active && s->active.size() + admit.size() >= s->max_active) break;
                used += need;
                admit.push_back(v);
                s->queue.pop_front();
            }
        }
        for (Served* v : admit) {
            const ecris_request& r = v->req->r;
            ecris_status st = take_slot(s, v) ? ECRIS_OK : ECRIS_ENOMEM;
            if (st == ECRIS_OK)
                st = ecris_batch_add_run(s->batch, &r.geo, &r.bf, &r.grid, &r.sp, &r.mcc, r.n, r.xyzv, r.q, r.weight,
                                         r.seed, r.dt, 0, &v->run);
            std::lock_guard<std::mutex> lock(s->mu);
            if (st != ECRIS_OK) {
                give_slot(s, v);
                finish(s, v, ECRIS_REQ_FAILED, ecris_batch_last_error(s->batch));
                if (v->job) calib_advance(s, v, false);
                ++s->n_done;
                continue;
            }
            v->res.state = ECRIS_REQ_RUNNING;
            v->res.t_admit = now_s(s);
            s->active.push_back(v);
            s->resident += (double)r.n;
        }
        // the launch shape for the resident mix: tuned again when the resident
        // particles have doubled or halved since the last tuning (the tuner
        // restores every run's state, so results are unaffected)
        if (!s->active.empty() && (s->tuned_at <= 0.0 || s->resident >= 2.0 * s->tuned_at ||
                                   s->resident <= 0.5 * s->tuned_at)) {
            if (ecris::batch_autotune(s->batch, 2, false, nullptr) == ECRIS_OK) {
                s->tuned_at = s->resident;
                std::lock_guard<std::mutex> lock(s->mu);
                ++s->n_tunes;
            }
        }
        // 2. one tick of the whole batch, and the snapshots at window boundaries
        std::vector<Served*> taken;
        if (!s->active.empty()) {
            if (ecris_batch_step(s->batch, s->steps_per_tick) != ECRIS_OK) {
                std::lock_guard<std::mutex> lock(s->mu);
                s->err = ecris_batch_last_error(s->batch);
                for (Served* v : s->active) {
                    finish(s, v, ECRIS_REQ_FAILED, s->err.c_str());
                    if (v->job) calib_advance(s, v, false);
                }
                s->n_done += (int64_t)s->active.size();
                s->active.clear();
                waiting.clear();
                continue;
            }
            double advanced = 0.0;
            for (Served* v : s->active) {
                const ecris_request& r = v->req->r;
                v->issued += s->steps_per_tick;
                advanced += (double)r.n * s->steps_per_tick;
                if (v->issued % r.window_steps == 0 &&
                    ecris::batch_snapshot(s->batch, v->run, v->snap) == ECRIS_OK &&
                    cudaEventRecord(v->ev, bs) == cudaSuccess) {
                    v->snap_steps = v->issued;
                    taken.push_back(v);
                }
                // self-consistent n_e: updated on the device after every
                // ne_windows windows, in stream order, as the same run alone
                // would be between its calls of that many windows
                if (r.ne_windows && v->issued % ((uint64_t)r.window_steps * r.ne_windows) == 0 &&
                    ecris_batch_update_ne(s->batch, v->run) != ECRIS_OK)
                    v->ne_failed = true;
            }
            std::lock_guard<std::mutex> lock(s->mu);
            s->ion_steps += advanced;
        }
        // 3. the previous tick's snapshots, read while this tick runs
        std::vector<std::pair<Served*, int32_t>> retire;
        for (Served* v : waiting) {
            const bool landed = cudaEventSynchronize(v->ev) == cudaSuccess;
            const ecris_request& r = v->req->r;
            ecris_result res;
            {
                std::lock_guard<std::mutex> lock(s->mu);
                res = v->res;
            }
            const bool ok_diag = landed && !v->ne_failed && read_snapshot(s, v, ext, res);
            const bool conv = ok_diag && converged(v, ext, res);
            const bool cap = v->snap_steps >= r.max_steps;
            res.converged = conv ? 1 : 0;
            {
                std::lock_guard<std::mutex> lock(s->mu);
                v->res = res;   // the result at this boundary, visible to poll
            }
            if (ok_diag && !conv && !cap) continue;
            retire.push_back({v, ok_diag ? ECRIS_REQ_DONE : ECRIS_REQ_FAILED});
        }
        for (auto& rv : retire) {
            Served* v = rv.first;
            // a snapshot of the run enqueued this tick must land before its slot is reused
            auto it = std::find(taken.begin(), taken.end(), v);
            if (it != taken.end()) {
                cudaEventSynchronize(v->ev);
                taken.erase(it);
            }
            ecris_batch_remove_run(s->batch, v->run);
            s->resident -= (double)v->req->r.n;
            give_slot(s, v);
            std::lock_guard<std::mutex> lock(s->mu);
            finish(s, v, rv.second,
                   rv.second == ECRIS_REQ_DONE ? nullptr
                   : v->ne_failed              ? "self-consistent n_e update failed"
                                               : "device error word set (bounded wait ran out)");
            if (v->job) calib_advance(s, v, rv.second == ECRIS_REQ_DONE);
            v->req.reset();   // the host copy of the inputs is no longer needed
            s->active.erase(std::find(s->active.begin(), s->active.end(), v));
            ++s->n_done;
        }
        waiting.swap(taken);
    }
}

template <class T>
void own(std::vector<T>& dst, const T* src, size_t n)
{
    if (src) dst.assign(src, src + n);
    else dst.clear();
}

// the checks of ecris_server_submit
ecris_status check_request(const ecris_server* s, const ecris_request& r, const char** why)
{
    if (r.window_steps == 0 || r.window_steps % s->steps_per_tick != 0 || r.max_steps == 0 ||
        r.max_steps % r.window_steps != 0 || !(r.dt > 0.0) || !(r.rel_tol > 0.0) || r.sp.qmax < 1 ||
        r.sp.qmax > 63 || r.grid.nx < 2 || r.grid.ny < 2 || r.grid.nz < 2) {
        *why = "server_submit: need window_steps a multiple of steps_per_tick, max_steps a multiple of "
               "window_steps, dt > 0, rel_tol > 0 and a valid species and mesh";
        return ECRIS_EINVAL;
    }
    if (r.n && (!r.q || !r.xyzv[0] || !r.xyzv[1] || !r.xyzv[2] || !r.xyzv[3] || !r.xyzv[4] || !r.xyzv[5])) {
        *why = "server_submit: NULL particle array";
        return ECRIS_EINVAL;
    }
    const size_t need = ecris_run_bytes(r.n, r.grid.nx, r.grid.ny, r.grid.nz, (r.mcc.flags & ECRIS_F_COULOMB) != 0);
    if (s->budget && need > s->budget) {
        *why = "server_submit: the run alone exceeds the memory budget";
        return ECRIS_ENOMEM;
    }
    return ECRIS_OK;
}

// a copy of the request with every array owned
std::unique_ptr<OwnedRequest> own_request(const ecris_request& r)
{
    auto o = std::make_unique<OwnedRequest>();
    o->r = r;
    const size_t nc = (size_t)r.grid.nx * r.grid.ny * r.grid.nz;
    own(o->E, r.grid.E, 3 * nc);
    own(o->ne_cells, r.grid.ne_in_cells, nc);
    own(o->ip, r.sp.ip_eV, (size_t)r.sp.qmax);
    own(o->axial, r.bf.B_axial, r.bf.n_axial > 0 ? (size_t)r.bf.n_axial : 0);
    own(o->nout, r.sp.n_outer, (size_t)r.sp.qmax);
    own(o->q, r.q, r.n);
    for (int k = 0; k < 6; ++k) own(o->xyzv[k], r.xyzv[k], r.n);
    o->r.grid.E = r.grid.E ? o->E.data() : nullptr;
    o->r.grid.ne_in_cells = r.grid.ne_in_cells ? o->ne_cells.data() : nullptr;
    o->r.sp.ip_eV = o->ip.data();
    o->r.bf.B_axial = r.bf.B_axial ? o->axial.data() : nullptr;
    o->r.sp.n_outer = o->nout.data();
    o->r.q = o->q.data();
    for (int k = 0; k < 6; ++k) o->r.xyzv[k] = o->xyzv[k].data();
    return o;
}

}  // namespace

extern "C" {

ecris_status ecris_server_create(ecris_server** out, int device, size_t hbm_budget_bytes, uint32_t steps_per_tick,
                                 uint32_t max_active)
{
    if (!out || steps_per_tick == 0) return ECRIS_EINVAL;
    *out = nullptr;
    ecris_server* s = new (std::nothrow) ecris_server();
    if (!s) return ECRIS_ENOMEM;
    s->device = device;
    s->budget = hbm_budget_bytes;
    s->steps_per_tick = steps_per_tick;
    s->max_active = max_active;
    const ecris_status st = ecris_batch_create(&s->batch, device, nullptr, hbm_budget_bytes);
    if (st != ECRIS_OK) {
        delete s;
        return st;
    }
    s->t0 = Clock::now();
    s->loop = std::thread(serve_loop, s);
    *out = s;
    return ECRIS_OK;
}

void ecris_server_destroy(ecris_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->loop.joinable()) s->loop.join();
    ecris_batch_destroy(s->batch);
    for (auto& kv : s->all) give_slot(s, kv.second.get());
    for (auto* p : s->free_snaps) cudaFreeHost(p);
    for (auto e : s->free_events) cudaEventDestroy(e);
    delete s;
}

const char* ecris_server_last_error(const ecris_server* s)
{
    return s ? s->err.c_str() : "";
}

ecris_status ecris_server_submit(ecris_server* s, const ecris_request* req, int64_t* ticket)
{
    if (!s) return ECRIS_EINVAL;
    auto fail = [s](ecris_status st, const char* msg) {
        std::lock_guard<std::mutex> lock(s->mu);
        s->err = msg;
        return st;
    };
    if (!req || !ticket) return fail(ECRIS_EINVAL, "server_submit: NULL argument");
    const char* why = nullptr;
    const ecris_status cst = check_request(s, *req, &why);
    if (cst != ECRIS_OK) return fail(cst, why);
    auto v = std::make_unique<Served>();
    auto o = own_request(*req);
    v->req = std::move(o);
    std::memset(&v->res, 0, sizeof v->res);
    v->res.state = ECRIS_REQ_QUEUED;
    std::lock_guard<std::mutex> lock(s->mu);
    v->ticket = s->next_ticket++;
    v->res.t_submit = now_s(s);
    *ticket = v->ticket;
    s->queue.push_back(v.get());
    s->all[v->ticket] = std::move(v);
    s->cv.notify_all();
    return ECRIS_OK;
}

ecris_status ecris_server_poll(ecris_server* s, int64_t ticket, ecris_result* out)
{
    if (!s || !out) return ECRIS_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) {
        s->err = "server_poll: unknown ticket";
        return ECRIS_EINVAL;
    }
    *out = it->second->res;
    return ECRIS_OK;
}

ecris_status ecris_server_stats(ecris_server* s, double* now, int64_t* queued, int64_t* running, int64_t* done,
                                double* ion_steps)
{
    if (!s) return ECRIS_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    if (now) *now = now_s(s);
    if (queued) *queued = (int64_t)s->queue.size();
    if (running) *running = (int64_t)s->active.size();
    if (done) *done = s->n_done;
    if (ion_steps) *ion_steps = s->ion_steps;
    return ECRIS_OK;
}

ecris_status ecris_server_tunings(ecris_server* s, int64_t* count)
{
    if (!s || !count) return ECRIS_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    *count = s->n_tunes;
    return ECRIS_OK;
}

ecris_status ecris_server_calibrate(ecris_server* s, const ecris_calib_request* req, int64_t* job)
{
    if (!s) return ECRIS_EINVAL;
    auto fail = [s](ecris_status st, const char* msg) {
        std::lock_guard<std::mutex> lock(s->mu);
        s->err = msg;
        return st;
    };
    if (!req || !job) return fail(ECRIS_EINVAL, "server_calibrate: NULL argument");
    if (!(req->flow_target > 0.0) || !(req->power_target_W > 0.0) || !(req->tol > 0.0) ||
        !std::isfinite(req->flow_target) || !std::isfinite(req->power_target_W) || req->max_iter < 1 ||
        req->max_iter > ECRIS_CALIB_HISTORY || !(req->base.weight > 0.0) || !(req->base.grid.Te_warm_eV > 0.0))
        return fail(ECRIS_EINVAL, "server_calibrate: need targets > 0, tol > 0, 1 <= max_iter <= "
                                  "ECRIS_CALIB_HISTORY, weight > 0 and T_ew > 0");
    const char* why = nullptr;
    const ecris_status cst = check_request(s, req->base, &why);
    if (cst != ECRIS_OK) return fail(cst, why);
    auto j = std::make_unique<CalibJob>();
    j->base = own_request(req->base);
    j->flow_target = req->flow_target;
    j->power_target = req->power_target_W;
    j->tol = req->tol;
    j->max_iter = req->max_iter;
    j->w = req->base.weight;
    j->Te = req->base.grid.Te_warm_eV;
    std::memset(&j->res, 0, sizeof j->res);
    j->res.state = ECRIS_REQ_RUNNING;
    std::lock_guard<std::mutex> lock(s->mu);
    j->id = s->next_job++;
    *job = j->id;
    auto v = calib_run(s, j.get());
    s->queue.push_back(v.get());
    s->all[v->ticket] = std::move(v);
    s->calibs[j->id] = std::move(j);
    s->cv.notify_all();
    return ECRIS_OK;
}

ecris_status ecris_server_calib_poll(ecris_server* s, int64_t job, ecris_calib_result* out)
{
    if (!s || !out) return ECRIS_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->calibs.find(job);
    if (it == s->calibs.end()) {
        s->err = "server_calib_poll: unknown job";
        return ECRIS_EINVAL;
    }
    *out = it->second->res;
    return ECRIS_OK;
}

}  // extern "C"
