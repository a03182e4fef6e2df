// serve_eigs: a batch of independent eigen-solves on mixed grids (declared
// in include/nsstab.h).
//
// The solves are grouped by (nx, ny, dt) into units, each a batched stepper
// with one member per solve (its own Reynolds number, cylinder diameter and
// base flow) driven by the lockstep Krylov-Schur driver.  A small pool of
// host threads runs the units, each on its own non-blocking CUDA stream, so
// the kernels of different grids share the GPU.  Admission is by device
// memory: a worker starts the next unit (largest grids first) only when the
// running units' estimated footprint plus its own stays within the budget;
// a unit that finishes releases its share and wakes the waiting workers.
// Every unit fits the budget alone (groups are split to make it so), so
// the queue always drains.
#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <exception>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "arnoldi.h"
#include "stepper.cuh"

namespace nsstab {
namespace {

struct Unit {
    int nx = 0, ny = 0;
    double dt = 0.0;
    std::vector<int> jobs;   // indices into the job list
    size_t bytes = 0;        // estimated device footprint
    int group = 0;
};

// Upper estimate of the device memory of one unit of k solves: per member
// the stepper's fields and spectra (at most 4 physical fields and 5 half
// spectra = 9 n values) and its parameter set's tables and base-derived
// fields (at most 8 n values), the Krylov basis (m+1 FP64 vectors), the
// Gram-Schmidt partial sums; once per unit the restart buffer (m vectors),
// twiddle tables and a fixed allowance for graphs and allocation rounding.
size_t unit_bytes(int nx, int ny, int precision, int k, int m) {
    const size_t n = (size_t)nx * ny;
    const size_t w = (precision == 32) ? 4 : 8;
    const size_t per_member = w * 17 * n + 8 * n * (size_t)(m + 1) + 8 * 152 * (size_t)(m + 1) + 4096;
    const size_t once = 8 * n * (size_t)m + 6 * 16 * (size_t)(nx + ny) + ((size_t)64 << 20);
    return (size_t)k * per_member + once;
}

struct Shared {
    std::mutex mu;
    std::condition_variable cv;
    std::vector<char> taken;
    size_t used = 0;
    std::string first_error;
};

}  // namespace

static int run_unit(const nsstab_config& base_cfg, const Unit& u, const nsstab_eig_job* jobs, int m, int nev,
                    double tol, int max_restarts, int nsteps, double t0, nsstab_eig_result* results) {
    const int k = (int)u.jobs.size();
    nsstab_config c = base_cfg;
    c.nx = u.nx;
    c.ny = u.ny;
    c.dt = u.dt;
    std::vector<double> Re(k), D(k);
    std::vector<const double*> base(k), v0(k);
    for (int i = 0; i < k; ++i) {
        const nsstab_eig_job& j = jobs[u.jobs[i]];
        Re[i] = j.Re;
        D[i] = j.cyl_D;
        base[i] = j.base;
        v0[i] = j.v0;
    }
    c.Re = Re[0];
    c.cyl_D = D[0];
    cudaStream_t s = nullptr;
    StepperBase* st = nullptr;
    std::vector<ArnoldiOut> outs(k);
    int rc = NSSTAB_OK;
    const cudaError_t es = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (es != cudaSuccess) {
        set_error(std::string("serve_eigs: cudaStreamCreateWithFlags: ") + cudaGetErrorString(es));
        rc = NSSTAB_ERR_CUDA;
    } else {
        st = make_stepper(c, k, Re.data(), D.data(), 1, s);
        rc = st->init();
        if (rc == NSSTAB_OK) rc = st->set_base_ptrs(base.data());
        if (rc == NSSTAB_OK)
            rc = arnoldi_batch_run(st, s, (long)u.nx * u.ny, v0.data(), m, nev, tol, max_restarts, nsteps, outs);
    }
    const double t_end = steady_seconds();
    for (int i = 0; i < k; ++i) {
        nsstab_eig_result& r = results[u.jobs[i]];
        r.group = u.group;
        if (rc < 0) {
            r.status = rc;
            r.latency_s = t_end - t0;
            continue;
        }
        const ArnoldiOut& o = outs[i];
        r.status = o.status;
        r.n_eig = o.n_eig;
        r.n_conv = o.n_conv;
        r.n_matvec = o.n_matvec;
        r.latency_s = (o.done_at > 0.0 ? o.done_at : t_end) - t0;
        for (int e = 0; e < o.n_eig && e < NSSTAB_SERVE_MAX_EIG; ++e) {
            r.eig_re[e] = o.mu[e].real();
            r.eig_im[e] = o.mu[e].imag();
            r.resid[e] = o.resid[e];
        }
    }
    delete st;   // synchronises the stream and frees the stepper's memory
    if (s) cudaStreamDestroy(s);
    return rc;
}

}  // namespace nsstab

using namespace nsstab;

static int serve_eigs_impl(const nsstab_config* cfg, int njobs, const nsstab_eig_job* jobs, int m, int nev,
                           double tol, int max_restarts, double T, long long mem_budget, int max_concurrent,
                           nsstab_eig_result* results, int* ngroups);

// No C++ exception (thread creation, host allocation) crosses the C ABI.
extern "C" int serve_eigs(const nsstab_config* cfg, int njobs, const nsstab_eig_job* jobs, int m, int nev,
                          double tol, int max_restarts, double T, long long mem_budget, int max_concurrent,
                          nsstab_eig_result* results, int* ngroups) {
    try {
        return serve_eigs_impl(cfg, njobs, jobs, m, nev, tol, max_restarts, T, mem_budget, max_concurrent, results,
                               ngroups);
    } catch (const std::exception& e) {
        set_error(std::string("serve_eigs: ") + e.what());
        return NSSTAB_ERR_OUT_OF_MEMORY;
    } catch (...) {
        set_error("serve_eigs: unexpected host exception");
        return NSSTAB_ERR_CUDA;
    }
}

// Checks every job, groups the jobs by (nx, ny, dt) (in order of first
// appearance; groups that do not fit the budget alone are split, and jobs
// that cannot fit at all are marked out of memory), largest grids first.
static int plan_units(const nsstab_config* cfg, int njobs, const nsstab_eig_job* jobs, int m, int nev, double tol,
                      int max_restarts, double T, long long mem_budget, nsstab_eig_result* results,
                      std::vector<int>& nsteps, std::vector<Unit>& units, size_t& budget, const char* who) {
    auto bad = [&](const std::string& msg) {
        set_error(std::string(who) + ": " + msg);
        return NSSTAB_ERR_INVALID_ARG;
    };
    if (!cfg || !jobs || !results) return bad("null argument");
    if (njobs < 1) return bad("need njobs >= 1");
    if (m < 2 || m > 1024) return bad("need 2 <= m <= 1024");
    if (nev < 1 || nev >= m || nev > NSSTAB_SERVE_MAX_EIG - 1)
        return bad("need 1 <= nev < m and nev <= NSSTAB_SERVE_MAX_EIG - 1");
    if (max_restarts < 0 || !(tol >= 0) || !(T > 0)) return bad("need max_restarts >= 0, tol >= 0, T > 0");
    nsteps.assign(njobs, 0);
    for (int i = 0; i < njobs; ++i) {
        const nsstab_eig_job& j = jobs[i];
        const std::string at = "job " + std::to_string(i) + ": ";
        if (!j.base || !j.v0) return bad(at + "null base or v0");
        nsstab_config c = *cfg;
        c.nx = j.nx;
        c.ny = j.ny;
        c.dt = j.dt;
        c.Re = j.Re;
        c.cyl_D = j.cyl_D;
        if (validate_config(c) != NSSTAB_OK) return bad(at + last_error());
        if ((long)j.nx * j.ny <= m) return bad(at + "need m < nx*ny");
        const double ns = T / j.dt, kk = std::round(ns);
        if (kk < 1 || std::fabs(ns - kk) > 1e-9 * std::max(1.0, ns) || kk > 1e9)
            return bad(at + "T must be a positive whole number of time steps");
        nsteps[i] = (int)kk;
    }
    std::memset(results, 0, sizeof(nsstab_eig_result) * (size_t)njobs);
    budget = (size_t)std::max<long long>(mem_budget, 0);
    if (mem_budget <= 0) {
        size_t fr = 0, tot = 0;
        NS_CUDA(cudaMemGetInfo(&fr, &tot));
        budget = (size_t)(0.8 * (double)fr);
    }
    std::map<std::tuple<int, int, double>, std::vector<int>> groups;
    std::vector<std::tuple<int, int, double>> order;
    for (int i = 0; i < njobs; ++i) {
        const auto key = std::make_tuple(jobs[i].nx, jobs[i].ny, jobs[i].dt);
        if (!groups.count(key)) order.push_back(key);
        groups[key].push_back(i);
    }
    int status = NSSTAB_OK;
    for (const auto& key : order) {
        const std::vector<int>& g = groups[key];
        const int nx = std::get<0>(key), ny = std::get<1>(key);
        int cap = (int)g.size();
        while (cap > 0 && unit_bytes(nx, ny, cfg->precision, cap, m) > budget) --cap;
        if (cap == 0) {
            for (int i : g) results[i].status = NSSTAB_ERR_OUT_OF_MEMORY;
            set_error(std::string(who) + ": a single solve on a " + std::to_string(nx) + "x" + std::to_string(ny) +
                      " grid exceeds the memory budget");
            status = NSSTAB_ERR_OUT_OF_MEMORY;
            continue;
        }
        cap = std::min(cap, 65535);
        for (size_t a = 0; a < g.size(); a += cap) {
            Unit u;
            u.nx = nx;
            u.ny = ny;
            u.dt = std::get<2>(key);
            u.jobs.assign(g.begin() + a, g.begin() + std::min(g.size(), a + (size_t)cap));
            u.bytes = unit_bytes(nx, ny, cfg->precision, (int)u.jobs.size(), m);
            units.push_back(u);
        }
    }
    std::stable_sort(units.begin(), units.end(),
                     [](const Unit& a, const Unit& b) { return (long)a.nx * a.ny > (long)b.nx * b.ny; });
    for (size_t i = 0; i < units.size(); ++i) units[i].group = (int)i;
    return status;
}

static int serve_eigs_impl(const nsstab_config* cfg, int njobs, const nsstab_eig_job* jobs, int m, int nev,
                           double tol, int max_restarts, double T, long long mem_budget, int max_concurrent,
                           nsstab_eig_result* results, int* ngroups) {
    std::vector<int> nsteps;
    std::vector<Unit> units;
    size_t budget = 0;
    int status = plan_units(cfg, njobs, jobs, m, nev, tol, max_restarts, T, mem_budget, results, nsteps, units,
                            budget, "serve_eigs");
    if (status == NSSTAB_ERR_INVALID_ARG || status == NSSTAB_ERR_CUDA) return status;
    int dev = 0;
    NS_CUDA(cudaGetDevice(&dev));
    const int workers_max = max_concurrent > 0 ? max_concurrent : 4;
    if (ngroups) *ngroups = (int)units.size();

    Shared sh;
    sh.taken.assign(units.size(), 0);
    const double t0 = steady_seconds();
    auto worker = [&]() {
        cudaSetDevice(dev);
        while (true) {
            int pick = -1;
            {
                std::unique_lock<std::mutex> lk(sh.mu);
                while (true) {
                    bool left = false;
                    for (size_t i = 0; i < units.size(); ++i) {
                        if (sh.taken[i]) continue;
                        left = true;
                        if (sh.used + units[i].bytes <= budget) {
                            pick = (int)i;
                            break;
                        }
                    }
                    if (pick >= 0 || !left) break;
                    sh.cv.wait(lk);
                }
                if (pick < 0) return;
                sh.taken[pick] = 1;
                sh.used += units[pick].bytes;
            }
            const Unit& u = units[pick];
            int rc;
            try {   // an exception must not end a worker thread (std::terminate)
                rc = run_unit(*cfg, u, jobs, m, nev, tol, max_restarts, nsteps[u.jobs[0]], t0, results);
            } catch (...) {
                set_error("serve_eigs: host exception while running a group");
                rc = NSSTAB_ERR_OUT_OF_MEMORY;
                for (int i : u.jobs) results[i].status = rc;
            }
            {
                std::lock_guard<std::mutex> lk(sh.mu);
                sh.used -= u.bytes;
                if (rc < 0 && sh.first_error.empty()) sh.first_error = last_error();
            }
            sh.cv.notify_all();
        }
    };
    const int nw = std::min<int>(workers_max, (int)units.size());
    std::vector<std::thread> pool;
    for (int w = 0; w < nw; ++w) pool.emplace_back(worker);
    for (auto& t : pool) t.join();

    if (!sh.first_error.empty()) set_error(sh.first_error);
    for (int i = 0; i < njobs; ++i) {
        const int s = results[i].status;
        if (s < 0 && status >= 0) status = s;
        if (s == NSSTAB_NOT_CONVERGED && status == NSSTAB_OK) status = s;
    }
    return status;
}

// ---------------------------------------------------------------- persistent

namespace nsstab {

// One wave of groups in one ragged stepper: every solve of the wave
// advanced by the same persistent launches, eigenproblems in lockstep rounds.
static int run_wave(const nsstab_config& base_cfg, const std::vector<const Unit*>& wave, const nsstab_eig_job* jobs,
                    const std::vector<int>& nsteps, int m, int nev, double tol, int max_restarts, double t0,
                    int wave_index, nsstab_eig_result* results) {
    cudaStream_t s = nullptr;
    NS_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    // released in reverse order on every exit, a host exception included:
    // the ragged launcher (which synchronises the stream and frees the
    // groups' memory) before its stream
    struct StreamOwner {
        cudaStream_t s;
        ~StreamOwner() { cudaStreamDestroy(s); }
    } stream_owner{s};
    std::unique_ptr<RaggedBase> rg(make_ragged_f32(s));
    std::vector<int> order;   // job index of each member
    int rc = NSSTAB_OK;
    for (const Unit* u : wave) {
        if (rc != NSSTAB_OK) break;
        const int k = (int)u->jobs.size();
        nsstab_config c = base_cfg;
        c.nx = u->nx;
        c.ny = u->ny;
        c.dt = u->dt;
        c.precision = 32;
        std::vector<double> Re(k), D(k);
        std::vector<const double*> base(k);
        for (int i = 0; i < k; ++i) {
            const nsstab_eig_job& j = jobs[u->jobs[i]];
            Re[i] = j.Re;
            D[i] = j.cyl_D;
            base[i] = j.base;
            order.push_back(u->jobs[i]);
        }
        c.Re = Re[0];
        c.cyl_D = D[0];
        rc = rg->add_group(c, k, Re.data(), D.data(), nsteps[u->jobs[0]], base.data());
    }
    if (rc == NSSTAB_OK) rc = rg->finalize();
    const int nb = (int)order.size();
    std::vector<ArnoldiOut> outs(nb);
    if (rc == NSSTAB_OK) {
        std::vector<long> nm(nb);
        std::vector<const double*> v0(nb);
        for (int b = 0; b < nb; ++b) {
            nm[b] = rg->n_of(b);
            v0[b] = jobs[order[b]].v0;
        }
        auto prod = [&](const double* const* in, double* const* out) { return rg->product(in, out); };
        rc = arnoldi_members_run(prod, nb, nm.data(), s, v0.data(), m, nev, tol, max_restarts, outs);
    }
    const double t_end = steady_seconds();
    for (int b = 0; b < nb; ++b) {
        nsstab_eig_result& r = results[order[b]];
        r.group = wave_index;
        if (rc < 0) {
            r.status = rc;
            r.latency_s = t_end - t0;
            continue;
        }
        const ArnoldiOut& o = outs[b];
        r.status = o.status;
        r.n_eig = o.n_eig;
        r.n_conv = o.n_conv;
        r.n_matvec = o.n_matvec;
        r.latency_s = (o.done_at > 0.0 ? o.done_at : t_end) - t0;
        for (int e = 0; e < o.n_eig && e < NSSTAB_SERVE_MAX_EIG; ++e) {
            r.eig_re[e] = o.mu[e].real();
            r.eig_im[e] = o.mu[e].imag();
            r.resid[e] = o.resid[e];
        }
    }
    return rc;
}

}  // namespace nsstab

static int serve_persistent_impl(const nsstab_config* cfg, int njobs, const nsstab_eig_job* jobs, int m, int nev,
                                 double tol, int max_restarts, double T, long long mem_budget,
                                 nsstab_eig_result* results, int* nwaves) {
    if (cfg && cfg->precision != 32) {
        set_error("serve_eigs_persistent: the persistent launch runs the FP32 stepper (precision 32)");
        return NSSTAB_ERR_INVALID_ARG;
    }
    std::vector<int> nsteps;
    std::vector<Unit> units;
    size_t budget = 0;
    int status = plan_units(cfg, njobs, jobs, m, nev, tol, max_restarts, T, mem_budget, results, nsteps, units,
                            budget, "serve_eigs_persistent");
    if (status == NSSTAB_ERR_INVALID_ARG || status == NSSTAB_ERR_CUDA) return status;
    // waves: groups in order (largest grids first) while their memory fits
    // the budget, at most kRagMaxGroups grids per launch
    const double t0 = steady_seconds();
    size_t next = 0;
    int waves = 0;
    std::string first_error;
    while (next < units.size()) {
        std::vector<const Unit*> wave;
        size_t used = 0;
        while (next < units.size() && (int)wave.size() < kRagMaxGroups &&
               (wave.empty() || used + units[next].bytes <= budget)) {
            used += units[next].bytes;
            wave.push_back(&units[next]);
            ++next;
        }
        const int rc = run_wave(*cfg, wave, jobs, nsteps, m, nev, tol, max_restarts, t0, waves, results);
        if (rc < 0 && first_error.empty()) first_error = last_error();
        ++waves;
    }
    if (nwaves) *nwaves = waves;
    if (!first_error.empty()) set_error(first_error);
    for (int i = 0; i < njobs; ++i) {
        const int s = results[i].status;
        if (s < 0 && status >= 0) status = s;
        if (s == NSSTAB_NOT_CONVERGED && status == NSSTAB_OK) status = s;
    }
    return status;
}

extern "C" int serve_eigs_persistent(const nsstab_config* cfg, int njobs, const nsstab_eig_job* jobs, int m, int nev,
                                     double tol, int max_restarts, double T, long long mem_budget,
                                     nsstab_eig_result* results, int* nwaves) {
    try {
        return serve_persistent_impl(cfg, njobs, jobs, m, nev, tol, max_restarts, T, mem_budget, results, nwaves);
    } catch (const std::exception& e) {
        set_error(std::string("serve_eigs_persistent: ") + e.what());
        return NSSTAB_ERR_OUT_OF_MEMORY;
    } catch (...) {
        set_error("serve_eigs_persistent: unexpected host exception");
        return NSSTAB_ERR_CUDA;
    }
}
