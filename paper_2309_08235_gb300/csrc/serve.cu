// serve.cu -- the serving loop behind priest_submit / priest_poll /
// priest_wait: continuous batching of planning requests (Alg. 1 per request)
// at the granularity of one CEM iteration.
//
// A worker thread owns the device side.  Each step it
//   1. admits queued requests while their buffers fit the HBM budget (one
//      device allocation handed out by a first-fit arena) and the slot limit,
//      in arrival order; a request whose robot still has a request on the
//      device waits for it, so a replan always starts from the finished
//      plan's state;
//   2. enqueues, on its own stream, one step for every admitted request: the
//      new requests' standard-normal draws (device stream, rng.cu) and setup
//      (one batched launch), then one persistent projection launch per
//      (dims, free-coefficient count) group over the samples of every
//      request -- each at its own CEM iteration -- and one batched
//      selection and refit launch over all of them;
//   3. while that step runs on the GPU, waits for the previous step and
//      completes the requests it finished: results are copied out, memory
//      returns to the arena and the tickets are released.
// Requests that arrive while others are on the GPU thus join the next step;
// every launch is shared by all requests resident at the time.
//
// Warm starts: a request with robot_id >= 0 keeps its sampling mean,
// covariance and final multipliers in a per-robot block of the arena.  The
// next request of the same robot with the same coefficient and sample counts
// starts from that mean / covariance, and its first projection starts from
// those multipliers (lambda^0 of the first CEM iteration); the last
// projection of every robot request writes them back.  Robot blocks are
// dropped least recently used first when memory is needed.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <tuple>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "arena.h"
#include "host_internal.h"

using namespace priest;
using namespace priest::host;

namespace priest {
namespace {

// Gathers of result words into one contiguous staging range.
struct CopyJob {
    const double *src;
    double *dst;
    int count;
};

__global__ void __launch_bounds__(128) gather_kernel(const CopyJob *jobs)
{
    const CopyJob j = jobs[blockIdx.x];
    for (int i = threadIdx.x; i < j.count; i += blockDim.x) j.dst[i] = j.src[i];
}

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    Shape sh;                            // resolved; obstacles ordered static first
    std::vector<double> center, vel, semi;
    uint64_t seed = 0;
    int64_t robot = -1;
    Clock::time_point t_submit;
    size_t bytes = 0;                    // device bytes of the request's own buffers
};

struct Robot {
    int D = 0, N = 0;
    size_t off = 0, bytes = 0;
    double *mu = nullptr, *cov = nullptr, *lam = nullptr;
    bool has_state = false;  // mu / cov / lam hold the robot's last successful plan
    bool busy = false;       // one of its requests is admitted and not yet completed
    uint64_t last_use = 0;
};

struct Slot {
    Request req;
    size_t off = 0;
    priest_loaded h;
    int *status = nullptr;
    Robot *robot = nullptr;
    bool warm = false;
    int l = 0;               // CEM iterations enqueued so far
    Tiling t{};
    size_t res_off = 0;      // offset of its results in the step's staging (finishing step)
};

size_t robot_bytes(int D, int N)
{
    return round_up(sizeof(double) * D) + round_up(sizeof(double) * D * D) + round_up(sizeof(double) * size_t(N) * D);
}

constexpr size_t kDefaultBudget = size_t(2) << 30;  // hbm_budget == 0

}  // namespace

struct Server {
    priest_ctx *ctx = nullptr;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, priest_result> done;
    std::unordered_set<uint64_t> outstanding;  // issued and not yet handed back
    uint64_t next_ticket = 1;
    bool stop = false;
    priest_serve_stats stats{};
    // device side (worker thread)
    cudaStream_t st = nullptr;
    char *arena_base = nullptr;
    Arena arena;
    std::unordered_map<int64_t, Robot> robots;
    uint64_t clock = 0;
    struct Stage {
        char *host = nullptr, *dev = nullptr;
        size_t host_bytes = 0, dev_bytes = 0;
        cudaEvent_t ev = nullptr;
        std::vector<Slot *> finishing;
        long trace_idx = -1;
        bool pending = false;
        cudaError_t err = cudaSuccess;
    } stage[2];
    bool fp32 = true;
    int L = 1;
    // optional step trace (environment variable PRIEST_SERVE_TRACE names a
    // file written when the context is destroyed): host times in ms since the
    // loop started, per step
    struct StepTrace {
        double t_begin, t_enqueued, t_done;
        int active, fresh, finishing;
    };
    bool trace_on = false;
    std::vector<StepTrace> trace;
    Clock::time_point t_origin;
    double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t_origin).count(); }

    void run();
    bool admit(std::unique_lock<std::mutex> &lk, std::vector<Slot *> &active, std::vector<Slot *> &fresh);
    bool alloc(size_t bytes, size_t *off);
    cudaError_t enqueue_step(std::vector<Slot *> &active, const std::vector<Slot *> &fresh, Stage &sg);
    template <typename Real>
    cudaError_t enqueue_step_t(std::vector<Slot *> &active, const std::vector<Slot *> &fresh, Stage &sg);
    void complete(Stage &sg);
    void finish_slot(Slot *s, const priest_result &res);
    cudaError_t grow(Stage &sg, size_t bytes);
    std::vector<char *> retired_host;
};

namespace {

// Byte layout of one step's staging block (identical on host and device).
struct StepLayout {
    size_t obs, init, setup, proj, items, cem, copies, counters, results, total;
};

}  // namespace

// Device memory for `bytes`, evicting least recently used idle robot blocks
// while it does not fit.
bool Server::alloc(size_t bytes, size_t *off)
{
    for (;;) {
        if (arena.alloc(bytes, off)) return true;
        auto victim = robots.end();
        for (auto it = robots.begin(); it != robots.end(); ++it)
            if (!it->second.busy && (victim == robots.end() || it->second.last_use < victim->second.last_use))
                victim = it;
        if (victim == robots.end()) return false;
        arena.release(victim->second.off, victim->second.bytes);
        robots.erase(victim);
        stats.evictions++;
    }
}

// Moves queued requests into slots (called with the queue lock held).
bool Server::admit(std::unique_lock<std::mutex> &, std::vector<Slot *> &active, std::vector<Slot *> &fresh)
{
    const int limit = ctx->cfg.serve_slots;
    for (auto it = queue.begin(); it != queue.end();) {
        if (limit > 0 && int(active.size() + fresh.size()) >= limit) break;
        Request &r = *it;
        Robot *rb = nullptr;
        if (r.robot >= 0) {
            auto f = robots.find(r.robot);
            if (f != robots.end()) {
                if (f->second.busy) {  // its previous request is still on the device
                    ++it;
                    continue;
                }
                rb = &f->second;
            }
        }
        // (the robot's own block is kept out of the eviction while room is made)
        if (rb) rb->busy = true;
        size_t off = 0;
        if (!alloc(r.bytes, &off)) {
            if (rb) rb->busy = false;
            stats.deferred++;
            break;
        }
        const int D = r.sh.D, N = r.sh.N;
        if (r.robot >= 0 && (!rb || rb->D != D || rb->N != N)) {
            if (rb) {  // shape changed: the old state cannot seed this request
                arena.release(rb->off, rb->bytes);
                robots.erase(r.robot);
                rb = nullptr;
            }
            size_t roff = 0;
            rb = nullptr;
            Robot fresh_rb;
            fresh_rb.bytes = robot_bytes(D, N);
            if (!alloc(fresh_rb.bytes, &roff)) {
                arena.release(off, r.bytes);
                stats.deferred++;
                break;
            }
            fresh_rb.D = D;
            fresh_rb.N = N;
            fresh_rb.off = roff;
            char *b = arena_base + roff;
            fresh_rb.mu = reinterpret_cast<double *>(b);
            fresh_rb.cov = reinterpret_cast<double *>(b + round_up(sizeof(double) * D));
            fresh_rb.lam = reinterpret_cast<double *>(b + round_up(sizeof(double) * D) + round_up(sizeof(double) * D * D));
            rb = &(robots[r.robot] = fresh_rb);
        }
        Slot *s = new Slot();
        s->req = std::move(r);
        it = queue.erase(it);
        s->off = off;
        const Carve k = carve(s->req.sh, fp32, L, false);
        s->h.sh = s->req.sh;
        carve_ptrs(&s->h, arena_base + off, k, fp32, L, false);
        s->h.bytes = k.total;
        s->status = reinterpret_cast<int *>(s->h.out + s->h.sh.D + 4);
        s->t = fp32 ? batch_tiling<float>(s->h.sh) : batch_tiling<double>(s->h.sh);
        if (rb) {
            s->robot = rb;
            rb->busy = true;
            rb->last_use = ++clock;
            s->warm = rb->has_state;
            // the robot block holds the request's mean and covariance
            s->h.mu = rb->mu;
            s->h.cov = rb->cov;
            if (s->warm) stats.warm_starts++;
        }
        s->h.default_mu = !s->warm;
        s->h.default_cov = !s->warm;
        fresh.push_back(s);
    }
    const size_t used = arena.used();
    if (used > stats.peak_bytes) stats.peak_bytes = used;
    return !fresh.empty();
}

// Grows a stage's staging block without a device-wide synchronisation: the
// device side is reallocated in stream order, the old pinned host block is
// retired (freed with the server).  The stage's previous step is complete
// when this is called.
cudaError_t Server::grow(Stage &sg, size_t bytes)
{
    if (bytes > sg.host_bytes) {
        if (sg.host) retired_host.push_back(sg.host);
        sg.host = nullptr;
        sg.host_bytes = 0;
        const size_t want = std::max(bytes, size_t(4) << 20) * 2;
        cudaError_t e = cudaHostAlloc(reinterpret_cast<void **>(&sg.host), want, cudaHostAllocDefault);
        if (e != cudaSuccess) return e;
        sg.host_bytes = want;
    }
    if (bytes > sg.dev_bytes) {
        if (sg.dev) cudaFreeAsync(sg.dev, st);
        sg.dev = nullptr;
        sg.dev_bytes = 0;
        const size_t want = std::max(bytes, size_t(4) << 20) * 2;
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&sg.dev), want, st);
        if (e != cudaSuccess) return e;
        sg.dev_bytes = want;
    }
    return cudaSuccess;
}

cudaError_t Server::enqueue_step(std::vector<Slot *> &active, const std::vector<Slot *> &fresh, Stage &sg)
{
    return fp32 ? enqueue_step_t<float>(active, fresh, sg) : enqueue_step_t<double>(active, fresh, sg);
}

template <typename Real>
cudaError_t Server::enqueue_step_t(std::vector<Slot *> &active, const std::vector<Slot *> &fresh, Stage &sg)
{
    // ---- groups of the projection launch: same dims, free-coefficient count
    //      and projection kernel
    std::map<std::tuple<int, int, int>, std::vector<Slot *>> groups;
    for (Slot *s : active) groups[{s->h.sh.dims, s->h.sh.nf, s->t.kind}].push_back(s);
    // ---- layout of the staging block
    StepLayout lay;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = round_up(o + bytes);
        return at;
    };
    size_t obs_bytes = 0;
    for (Slot *s : fresh) obs_bytes += sizeof(double) * (2 * s->req.center.size() + s->req.semi.size());
    size_t n_items = 0;
    for (auto &g : groups)
        for (Slot *s : g.second) n_items += (s->h.sh.N + s->t.S - 1) / s->t.S;
    sg.finishing.clear();
    size_t res_doubles = 0;
    for (Slot *s : active)
        if (s->l == L - 1) {
            sg.finishing.push_back(s);
            res_doubles += 2 * size_t(s->h.sh.D) + 5;
        }
    lay.obs = take(obs_bytes);
    lay.init = take(sizeof(GaussJob) * fresh.size());
    lay.setup = take(sizeof(SetupParams) * fresh.size());
    lay.proj = take(sizeof(ProjParams<Real>) * active.size());
    lay.items = take(sizeof(int2) * n_items);
    lay.cem = take(sizeof(CemArgs) * active.size());
    lay.copies = take(sizeof(CopyJob) * 2 * sg.finishing.size());
    lay.counters = take(sizeof(int) * groups.size());
    lay.results = take(sizeof(double) * res_doubles);
    lay.total = o;
    cudaError_t e = grow(sg, lay.total);
    if (e != cudaSuccess) return e;
    char *H = sg.host, *Dv = sg.dev;
    const size_t upload = lay.results;  // everything before the results is uploaded

    // ---- new requests: obstacles, draws + status / counter reset, setup
    GaussJob *jobs = reinterpret_cast<GaussJob *>(H + lay.init);
    SetupParams *sps = reinterpret_cast<SetupParams *>(H + lay.setup);
    size_t ob = lay.obs, smem_setup = 0;
    long long max_count = 0;
    for (size_t i = 0; i < fresh.size(); ++i) {
        Slot *s = fresh[i];
        priest_loaded h = s->h;  // setup reads the obstacles from the staging block
        const size_t nc = s->req.center.size(), ns = s->req.semi.size();
        std::memcpy(H + ob, s->req.center.data(), sizeof(double) * nc);
        h.center = reinterpret_cast<double *>(Dv + ob);
        ob += sizeof(double) * nc;
        std::memcpy(H + ob, s->req.vel.data(), sizeof(double) * nc);
        h.vel = reinterpret_cast<double *>(Dv + ob);
        ob += sizeof(double) * nc;
        std::memcpy(H + ob, s->req.semi.data(), sizeof(double) * ns);
        h.semi = reinterpret_cast<double *>(Dv + ob);
        ob += sizeof(double) * ns;
        sps[i] = setup_params(ctx, &h, true, s->status);
        smem_setup = std::max(smem_setup, setup_smem_bytes(s->h.sh));
        const long long cnt = (long long)L * s->h.sh.N * s->h.sh.D;
        jobs[i].seed = s->req.seed;
        jobs[i].count = cnt;
        jobs[i].out = s->h.z;
        jobs[i].status = s->status;
        jobs[i].counter = s->h.counter;
        max_count = std::max(max_count, cnt);
    }
    // ---- projection parameters and items, group by group
    ProjParams<Real> *pp = reinterpret_cast<ProjParams<Real> *>(H + lay.proj);
    int2 *items = reinterpret_cast<int2 *>(H + lay.items);
    struct GroupLaunch {
        int dims, nf, nv, want_lambda, kind, R;
        size_t first_param, first_item, n_items, smem;
    };
    std::vector<GroupLaunch> launches;
    size_t np = 0, ni = 0;
    for (auto &g : groups) {
        GroupLaunch gl{std::get<0>(g.first), std::get<1>(g.first), g.second.front()->h.sh.nv, 0, std::get<2>(g.first),
                       g.second.front()->t.R, np, ni, 0, 0};
        std::vector<std::pair<double, int2>> its;
        for (Slot *s : g.second) {
            const Shape &sh = s->h.sh;
            ProjParams<Real> p = proj_params<Real>(ctx, &s->h, s->t);
            p.N = sh.N;
            p.mode = 1;
            p.mu = s->h.mu;
            p.Lc = s->h.L;
            p.z = s->h.z + size_t(s->l) * sh.N * sh.D;
            const bool warm_lam = s->warm && s->l == 0;
            const bool write_lam = s->robot && s->l == L - 1;
            p.lam_in = warm_lam ? s->robot->lam : nullptr;
            p.lam_out = write_lam ? s->robot->lam : nullptr;
            p.want_lambda = write_lam ? 1 : 0;
            p.xi_bar = s->h.xb;
            p.r_out = s->h.r;
            p.c1_out = s->h.c1;
            gl.want_lambda |= p.want_lambda;
            gl.smem = std::max(gl.smem, s->t.smem);
            const int idx = int(np - gl.first_param);
            pp[np++] = p;
            const double cost = double(sh.n_p) * (double(sh.n_obs) + 12.0);
            for (int s0 = 0; s0 < sh.N; s0 += s->t.S)
                its.push_back({cost * std::min(s->t.S, sh.N - s0), make_int2(idx, s0)});
        }
        std::stable_sort(its.begin(), its.end(), [](const std::pair<double, int2> &a, const std::pair<double, int2> &b) {
            return a.first > b.first;
        });
        for (auto &x : its) items[ni++] = x.second;
        gl.n_items = ni - gl.first_item;
        launches.push_back(gl);
    }
    // ---- selection / refit arguments, in the order of the parameters above
    CemArgs *cem = reinterpret_cast<CemArgs *>(H + lay.cem);
    size_t nc = 0, smem_select = 0, smem_refit = 0;
    int D_max = 0;
    for (auto &g : groups)
        for (Slot *s : g.second) {
            cem[nc++] = cem_args(ctx, &s->h, s->status, s->h.out);
            smem_select = std::max(smem_select, select_smem_bytes(s->h.sh.N));
            smem_refit = std::max(smem_refit, refit_smem_bytes(s->h.sh.D, s->h.sh.n_elite));
            D_max = std::max(D_max, s->h.sh.D);
        }
    // ---- result gathers of the requests that finish in this step
    CopyJob *cj = reinterpret_cast<CopyJob *>(H + lay.copies);
    size_t ro = lay.results, nj = 0;
    for (Slot *s : sg.finishing) {
        const int D = s->h.sh.D;
        s->res_off = ro;
        cj[nj++] = CopyJob{s->h.out, reinterpret_cast<double *>(Dv + ro), D + 5};
        ro += sizeof(double) * (D + 5);
        cj[nj++] = CopyJob{s->h.mu, reinterpret_cast<double *>(Dv + ro), D};
        ro += sizeof(double) * D;
    }
    std::memset(H + lay.counters, 0, sizeof(int) * groups.size());

    // ---- the step's launches
    e = cudaMemcpyAsync(Dv, H, upload, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    if (!fresh.empty()) {
        e = launch_normal_batch(reinterpret_cast<const GaussJob *>(Dv + lay.init), int(fresh.size()), max_count, st);
        if (e == cudaSuccess)
            e = launch_setup_batch(reinterpret_cast<const SetupParams *>(Dv + lay.setup), int(fresh.size()), smem_setup,
                                   st);
        ctx->launches += 2;
        if (e != cudaSuccess) return e;
        for (Slot *s : fresh) s->h.shape_ready = true;
    }
    const ProjParams<Real> *ppd = reinterpret_cast<const ProjParams<Real> *>(Dv + lay.proj);
    const int2 *itd = reinterpret_cast<const int2 *>(Dv + lay.items);
    int *cnt = reinterpret_cast<int *>(Dv + lay.counters);
    for (size_t gi = 0; gi < launches.size(); ++gi) {
        const GroupLaunch &gl = launches[gi];
        e = launch_project_batch<Real>(ppd + gl.first_param, itd + gl.first_item, int(gl.n_items), cnt + gi, gl.dims,
                                       gl.R, 0, gl.nf, gl.nv, gl.want_lambda, gl.smem, 0, st, gl.kind);
        ctx->launches++;
        if (e != cudaSuccess) return e;
    }
    const CemArgs *cemd = reinterpret_cast<const CemArgs *>(Dv + lay.cem);
    e = launch_select_batch(cemd, int(active.size()), smem_select, st);
    if (e == cudaSuccess) e = launch_refit_batch(cemd, int(active.size()), D_max, smem_refit, st);
    ctx->launches += 2;
    if (e != cudaSuccess) return e;
    if (!sg.finishing.empty()) {
        gather_kernel<<<unsigned(nj), 128, 0, st>>>(reinterpret_cast<const CopyJob *>(Dv + lay.copies));
        ctx->launches++;
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(H + lay.results, Dv + lay.results, ro - lay.results, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return e;
    }
    for (Slot *s : active) s->l++;
    return cudaEventRecord(sg.ev, st);
}

void Server::finish_slot(Slot *s, const priest_result &res)
{
    if (s->robot) {
        s->robot->busy = false;
        s->robot->has_state = res.status == PRIEST_OK;
        s->robot->last_use = ++clock;
    }
    arena.release(s->off, s->req.bytes);
    {
        std::lock_guard<std::mutex> lk(mu);
        done[s->req.ticket] = res;
        stats.completed++;
    }
    delete s;
}

// Waits for a step and completes the requests that finished in it.
void Server::complete(Stage &sg)
{
    if (!sg.pending) return;
    sg.pending = false;
    cudaError_t e = sg.err;
    if (e != cudaSuccess)
        cudaStreamSynchronize(st);  // launches enqueued before the failure may still use the memory
    else
        e = cudaEventSynchronize(sg.ev);
    sg.err = cudaSuccess;
    const auto now = Clock::now();
    if (trace_on && sg.trace_idx >= 0) trace[size_t(sg.trace_idx)].t_done = now_ms();
    sg.trace_idx = -1;
    for (Slot *s : sg.finishing) {
        priest_result res;
        std::memset(&res, 0, sizeof(res));
        if (e == cudaSuccess) {
            const double *out = reinterpret_cast<const double *>(sg.host + s->res_off);
            const int D = s->h.sh.D;
            fill_result(s->h.sh, out, out + D + 5, &res);
            int status_word = 0;
            std::memcpy(&status_word, out + D + 4, sizeof(int));
            if (status_word) res.status = PRIEST_ERR_NUMERIC;
        } else {
            res.status = PRIEST_ERR_CUDA;
            res.D = s->h.sh.D;
        }
        res.latency_ms = std::chrono::duration<double, std::milli>(now - s->req.t_submit).count();
        finish_slot(s, res);
    }
    sg.finishing.clear();
    cv_done.notify_all();
}

void Server::run()
{
    cudaSetDevice(ctx->device);
    std::vector<Slot *> active;
    int cur = 0;
    for (;;) {
        std::vector<Slot *> fresh;
        {
            std::unique_lock<std::mutex> lk(mu);
            const bool idle = active.empty() && !stage[0].pending && !stage[1].pending;
            if (idle) cv_work.wait(lk, [&] { return stop || !queue.empty(); });
            if (stop) break;
            admit(lk, active, fresh);
            stats.submitted = int64_t(next_ticket - 1);
        }
        active.insert(active.end(), fresh.begin(), fresh.end());
        Stage &sg = stage[cur];
        if (!active.empty()) {
            const double t_begin = trace_on ? now_ms() : 0.0;
            const cudaError_t e = enqueue_step(active, fresh, sg);
            sg.pending = true;
            if (trace_on) {
                sg.trace_idx = long(trace.size());
                trace.push_back({t_begin, now_ms(), 0.0, int(active.size()), int(fresh.size()),
                                 int(sg.finishing.size())});
            }
            if (e != cudaSuccess) {
                // the whole step failed: every resident request reports it
                cudaGetLastError();
                sg.err = e;
                sg.finishing = active;
                active.clear();
            } else {
                std::lock_guard<std::mutex> lk(mu);
                stats.steps++;
                stats.slot_steps += int64_t(active.size());
                stats.max_active = std::max<int64_t>(stats.max_active, int64_t(active.size()));
            }
            // requests in their last iteration leave the resident set now;
            // their memory returns when the step is complete
            active.erase(std::remove_if(active.begin(), active.end(), [&](Slot *s) { return s->l >= L; }),
                         active.end());
        }
        complete(stage[cur ^ 1]);
        if (active.empty()) complete(sg);
        cur ^= 1;
    }
    // stop: let queued work go, finish what is on the device
    cudaStreamSynchronize(st);
    complete(stage[0]);
    complete(stage[1]);
    for (Slot *s : active) {
        priest_result res;
        std::memset(&res, 0, sizeof(res));
        res.status = PRIEST_ERR_CUDA;
        finish_slot(s, res);
    }
}

}  // namespace priest

namespace priest {
namespace host {

void server_destroy(priest_ctx *ctx)
{
    Server *sv = ctx->server;
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    if (sv->trace_on) {
        if (FILE *f = fopen(getenv("PRIEST_SERVE_TRACE"), "w")) {
            fprintf(f, "t_begin_ms,t_enqueued_ms,t_done_ms,active,fresh,finishing\n");
            for (const auto &t : sv->trace)
                fprintf(f, "%.3f,%.3f,%.3f,%d,%d,%d\n", t.t_begin, t.t_enqueued, t.t_done, t.active, t.fresh,
                        t.finishing);
            fclose(f);
        }
    }
    if (sv->st) cudaStreamSynchronize(sv->st);
    for (auto &sg : sv->stage) {
        if (sg.ev) cudaEventDestroy(sg.ev);
        if (sg.host) cudaFreeHost(sg.host);
        if (sg.dev) cudaFreeAsync(sg.dev, sv->st);
    }
    for (char *h : sv->retired_host) cudaFreeHost(h);
    if (sv->st) cudaStreamSynchronize(sv->st);
    if (sv->arena_base) cudaFree(sv->arena_base);
    if (sv->st) cudaStreamDestroy(sv->st);
    delete sv;
    ctx->server = nullptr;
}

}  // namespace host
}  // namespace priest

namespace {

// Starts the serving loop on first use.
priest_status ensure_server(priest_ctx *ctx, Server **out)
{
    std::lock_guard<std::mutex> lk(ctx->server_mu);
    if (ctx->server) {
        *out = ctx->server;
        return PRIEST_OK;
    }
    Server *sv = new (std::nothrow) Server();
    if (!sv) return fail(ctx, PRIEST_ERR_NOMEM, "host allocation failed");
    sv->ctx = ctx;
    sv->fp32 = ctx->cfg.precision != PRIEST_FP64_CHECK;
    sv->L = ctx->cfg.cem_iters;
    const size_t budget = ctx->cfg.hbm_budget ? ctx->cfg.hbm_budget : kDefaultBudget;
    cudaError_t e = cudaStreamCreateWithFlags(&sv->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&sv->arena_base), budget);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&sv->stage[i].ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->server = sv;
        server_destroy(ctx);
        return fail(ctx, PRIEST_ERR_NOMEM, std::string("serving buffers: ") + cudaGetErrorString(e));
    }
    sv->arena.reset(budget, 256);
    sv->trace_on = getenv("PRIEST_SERVE_TRACE") != nullptr;
    sv->t_origin = Clock::now();
    sv->stats.budget_bytes = sv->arena.capacity();
    ctx->server = sv;
    sv->worker = std::thread([sv] { sv->run(); });
    *out = sv;
    return PRIEST_OK;
}

}  // namespace

extern "C" {

priest_status priest_submit(priest_ctx *ctx, const priest_problem *pr, uint64_t *ticket)
{
    if (!ctx || !ticket) return PRIEST_ERR_INVALID;
    Request req;
    std::string why;
    priest_status s = resolve(ctx->cfg, pr, -1, req.sh, why);
    if (s != PRIEST_OK) return fail(ctx, s, why);
    const bool fp32 = ctx->cfg.precision != PRIEST_FP64_CHECK;
    req.bytes = carve(req.sh, fp32, ctx->cfg.cem_iters, false).total;
    order_obstacles(req.sh, pr->center, pr->vel, pr->semi, req.center, req.vel, req.semi, req.sh.n_static);
    req.seed = pr->seed;
    req.robot = pr->robot_id >= 0 ? pr->robot_id : -1;
    const size_t need = req.bytes + (req.robot >= 0 ? robot_bytes(req.sh.D, req.sh.N) : 0);
    const size_t budget = ctx->cfg.hbm_budget ? ctx->cfg.hbm_budget : kDefaultBudget;
    if (need + 1024 > budget) return fail(ctx, PRIEST_ERR_BUDGET, "request larger than the HBM budget");
    Server *sv = nullptr;
    s = ensure_server(ctx, &sv);
    if (s != PRIEST_OK) return s;
    req.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        req.ticket = sv->next_ticket++;
        *ticket = req.ticket;
        sv->outstanding.insert(req.ticket);
        sv->queue.push_back(std::move(req));
    }
    sv->cv_work.notify_all();
    return PRIEST_OK;
}

priest_status priest_poll(priest_ctx *ctx, uint64_t ticket, priest_result *out)
{
    if (!ctx || !out) return PRIEST_ERR_INVALID;
    Server *sv = ctx->server;
    if (!sv) return PRIEST_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (!sv->outstanding.count(ticket)) return PRIEST_ERR_INVALID;
    auto it = sv->done.find(ticket);
    if (it == sv->done.end()) return PRIEST_PENDING;
    *out = it->second;
    sv->done.erase(it);
    sv->outstanding.erase(ticket);
    return PRIEST_OK;
}

priest_status priest_wait(priest_ctx *ctx, uint64_t ticket, double timeout_ms, priest_result *out)
{
    if (!ctx || !out) return PRIEST_ERR_INVALID;
    Server *sv = ctx->server;
    if (!sv) return PRIEST_ERR_INVALID;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (!sv->outstanding.count(ticket)) return PRIEST_ERR_INVALID;
    const auto ready = [&] { return sv->done.count(ticket) != 0; };
    if (timeout_ms < 0) {
        sv->cv_done.wait(lk, ready);
    } else if (!sv->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), ready)) {
        return PRIEST_ERR_TIMEOUT;
    }
    auto it = sv->done.find(ticket);
    *out = it->second;
    sv->done.erase(it);
    sv->outstanding.erase(ticket);
    return PRIEST_OK;
}

priest_status priest_serve_stats_get(priest_ctx *ctx, priest_serve_stats *out)
{
    if (!ctx || !out) return PRIEST_ERR_INVALID;
    std::memset(out, 0, sizeof(*out));
    Server *sv = ctx->server;
    if (!sv) return PRIEST_OK;
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->stats;
    out->submitted = int64_t(sv->next_ticket - 1);
    return PRIEST_OK;
}

}  // extern "C"
