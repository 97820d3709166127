// Several wavenumbers on one mesh (a frequency sweep, Section V): one plan
// per wavenumber, admitted to the device by an estimate of its memory, and
// the products of all admitted plans run as parallel branches of one CUDA
// graph.  The paper sweeps frequencies one after another; here the plans of
// a sweep share the GPU.
#include "../../include/mlfma.h"
#include "device.h"
#include "plan_host.h"

#include <algorithm>
#include <map>
#include <string>
#include <tuple>
#include <vector>

namespace mlfma {
void set_last_error(const std::string &msg);
int64_t plan_device_bytes_estimate(const PlanHost &H, const mlfma_opts &o);
int64_t plan_device_bytes(mlfma_plan_t p);
const PlanHost *plan_host(mlfma_plan_t p);
mlfma_status plan_attach_device(mlfma_plan_t p, const mlfma_opts &o);
void plan_detach_device(mlfma_plan_t p);
mlfma_status plan_enqueue_core(mlfma_plan_t p, int prec, int64_t Bi, cudaEvent_t fork, cudaEvent_t *done);
mlfma_status plan_enqueue_io(mlfma_plan_t p, int prec, const void *x, int xc, void *y, int64_t B, int finalize,
                             cudaStream_t s);
}  // namespace mlfma

using namespace mlfma;

struct mlfma_set_s {
    std::vector<double> ks;
    std::vector<mlfma_plan_t> plans;     // host tables always; device half while admitted
    std::vector<int64_t> est;            // estimated peak device bytes per plan
    std::vector<int> wave;               // admission wave of each plan
    int nwave = 0, resident = -1;        // the wave whose plans are on the device
    mlfma_opts opts{};
    int64_t budget = 0, n = 0;
    int device = 0;
    cudaStream_t cap = nullptr;
    cudaEvent_t fork = nullptr;
    std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;   // (wave, prec, columns)
};

namespace {

mlfma_status fail(mlfma_status st, const std::string &msg)
{
    set_last_error(msg);
    return st;
}

mlfma_status cuda_fail(cudaError_t e, const char *where)
{
    set_last_error(std::string(where) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MLFMA_ENOMEM : MLFMA_ECUDA;
}

void drop_graphs(mlfma_set_s *s)
{
    for (auto &kv : s->graphs) cudaGraphExecDestroy(kv.second);
    s->graphs.clear();
}

// Puts wave w on the device (taking the previous wave off first).
mlfma_status admit(mlfma_set_s *s, int w)
{
    if (s->resident == w) return MLFMA_OK;
    for (size_t f = 0; f < s->plans.size(); ++f)
        if (s->wave[f] == s->resident) plan_detach_device(s->plans[f]);
    s->resident = -1;
    for (size_t f = 0; f < s->plans.size(); ++f) {
        if (s->wave[f] != w) continue;
        mlfma_status st = plan_attach_device(s->plans[f], s->opts);
        if (st != MLFMA_OK) {
            for (size_t g = 0; g < f; ++g)
                if (s->wave[g] == w) plan_detach_device(s->plans[g]);
            return st;
        }
    }
    s->resident = w;
    return MLFMA_OK;
}

// All cores of wave w as parallel branches of one graph: fork from one
// event on the capture stream, join every plan's completion back.
mlfma_status wave_graph(mlfma_set_s *s, int w, int prec, int64_t Bi, cudaGraphExec_t *out)
{
    auto key = std::make_tuple(w, prec, (int)Bi);
    auto it = s->graphs.find(key);
    if (it != s->graphs.end()) {
        *out = it->second;
        return MLFMA_OK;
    }
    cudaError_t e = cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "set graph capture");
    mlfma_status st = MLFMA_OK;
    if ((e = cudaEventRecord(s->fork, s->cap)) != cudaSuccess) st = cuda_fail(e, "set fork");
    for (size_t f = 0; f < s->plans.size() && st == MLFMA_OK; ++f) {
        if (s->wave[f] != w) continue;
        cudaEvent_t done = nullptr;
        st = plan_enqueue_core(s->plans[f], prec, Bi, s->fork, &done);
        if (st == MLFMA_OK && (e = cudaStreamWaitEvent(s->cap, done, 0)) != cudaSuccess) st = cuda_fail(e, "set join");
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s->cap, &g);
    if (st != MLFMA_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "set graph capture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "set graph instantiate");
    s->graphs[key] = ex;
    *out = ex;
    return MLFMA_OK;
}

class DeviceGuard {
  public:
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev_);
        if (dev != prev_) {
            cudaSetDevice(dev);
            set_ = true;
        }
    }
    ~DeviceGuard()
    {
        if (set_) cudaSetDevice(prev_);
    }

  private:
    int prev_ = 0;
    bool set_ = false;
};

}  // namespace

extern "C" {

mlfma_status mlfma_set_create(const double *verts, int64_t nv, const int32_t *tris, int64_t nt, const double *ks,
                              int nk, int levels, double digits, const mlfma_opts *opts, int64_t budget_bytes,
                              mlfma_set_t *out)
{
    if (!out || !ks || nk < 1) return fail(MLFMA_EINVAL, "out or ks is NULL, or nk < 1");
    mlfma_set_s *s = new (std::nothrow) mlfma_set_s();
    if (!s) return fail(MLFMA_ENOMEM, "host allocation failed");
    if (opts) s->opts = *opts; else mlfma_default_opts(&s->opts);
    s->opts.host_only = 0;
    int dev = s->opts.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        delete s;
        return fail(MLFMA_ECUDA, "cudaGetDevice failed");
    }
    s->device = dev;
    s->opts.device = dev;
    mlfma_opts host = s->opts;
    host.host_only = 1;
    for (int f = 0; f < nk; ++f) {
        mlfma_plan_t p = nullptr;
        mlfma_status st = mlfma_plan(verts, nv, tris, nt, ks[f], levels, digits, &host, &p);
        if (st != MLFMA_OK) {
            mlfma_set_destroy(s);
            return st;
        }
        s->ks.push_back(ks[f]);
        s->plans.push_back(p);
        s->est.push_back(plan_device_bytes_estimate(*plan_host(p), s->opts));
    }
    s->n = plan_host(s->plans[0])->N;
    DeviceGuard g(dev);
    if (budget_bytes <= 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            mlfma_set_destroy(s);
            return fail(MLFMA_ECUDA, "cudaMemGetInfo failed");
        }
        budget_bytes = (int64_t)(0.9 * (double)fr);
    }
    s->budget = budget_bytes;
    // waves in wavenumber order, each as many plans as the budget holds
    int64_t used = 0;
    int w = 0;
    for (int f = 0; f < nk; ++f) {
        if (s->est[f] > budget_bytes) {
            const std::string msg = "plan for k = " + std::to_string(ks[f]) + " needs about " +
                                    std::to_string(s->est[f] >> 20) + " MiB; the admission budget is " +
                                    std::to_string(budget_bytes >> 20) + " MiB";
            mlfma_set_destroy(s);
            return fail(MLFMA_ENOMEM, msg);
        }
        if (used + s->est[f] > budget_bytes) {
            ++w;
            used = 0;
        }
        used += s->est[f];
        s->wave.push_back(w);
    }
    s->nwave = w + 1;
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming)) != cudaSuccess) {
        mlfma_set_destroy(s);
        return cuda_fail(e, "set streams");
    }
    mlfma_status st = admit(s, 0);
    if (st != MLFMA_OK) {
        mlfma_set_destroy(s);
        return st;
    }
    *out = s;
    return MLFMA_OK;
}

mlfma_status mlfma_set_info(mlfma_set_t s, int *nk, int *waves, int *wave_of, int64_t *est_bytes,
                            int64_t *device_bytes)
{
    if (!s) return fail(MLFMA_EINVAL, "set is NULL");
    if (nk) *nk = (int)s->plans.size();
    if (waves) *waves = s->nwave;
    for (size_t f = 0; f < s->plans.size(); ++f) {
        if (wave_of) wave_of[f] = s->wave[f];
        if (est_bytes) est_bytes[f] = s->est[f];
        if (device_bytes) device_bytes[f] = plan_device_bytes(s->plans[f]);
    }
    return MLFMA_OK;
}

mlfma_status mlfma_set_plan(mlfma_set_t s, int f, mlfma_plan_t *plan)
{
    if (!s || !plan || f < 0 || f >= (int)s->plans.size()) return fail(MLFMA_EINVAL, "bad set, index or out pointer");
    *plan = s->plans[f];
    return MLFMA_OK;
}

mlfma_status mlfma_set_matvec(mlfma_set_t s, const void *x, int x_shared, int xc, void *y, int64_t B, int prec,
                              void *stream)
{
    if (!s) return fail(MLFMA_EINVAL, "set is NULL");
    if (!x || !y) return fail(MLFMA_EINVAL, "x or y is NULL");
    if (B < 1 || B * (xc ? 2 : 1) > s->opts.max_batch) return fail(MLFMA_EINVAL, "B exceeds max_batch");
    if (prec != MLFMA_FP32 && prec != MLFMA_FP64) return fail(MLFMA_EINVAL, "unknown precision");
    if (!(s->opts.precisions & (1 << prec))) return fail(MLFMA_EINVAL, "precision not set up in the set");
    DeviceGuard g(s->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t Bi = B * (xc ? 2 : 1);
    const size_t rsz = prec == MLFMA_FP64 ? 8 : 4;
    const size_t xstride = x_shared ? 0 : (size_t)s->n * B * (xc ? 2 : 1) * rsz;
    const size_t ystride = (size_t)s->n * B * 2 * rsz;
    for (int w = 0; w < s->nwave; ++w) {
        if (s->resident != w) {
            // the device memory of the previous wave is released: its work must be done
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e, "set wave");
            drop_graphs(s);
            mlfma_status a = admit(s, w);
            if (a != MLFMA_OK) return a;
        }
        cudaGraphExec_t ex;
        mlfma_status r = wave_graph(s, w, prec, Bi, &ex);
        if (r != MLFMA_OK) return r;
        for (size_t f = 0; f < s->plans.size(); ++f)
            if (s->wave[f] == w &&
                (r = plan_enqueue_io(s->plans[f], prec, static_cast<const char *>(x) + f * xstride, xc, nullptr, B,
                                     0, st)) != MLFMA_OK)
                return r;
        cudaError_t e = cudaGraphLaunch(ex, st);
        if (e != cudaSuccess) return cuda_fail(e, "set graph launch");
        for (size_t f = 0; f < s->plans.size(); ++f)
            if (s->wave[f] == w &&
                (r = plan_enqueue_io(s->plans[f], prec, nullptr, xc, static_cast<char *>(y) + f * ystride, B, 1,
                                     st)) != MLFMA_OK)
                return r;
    }
    return MLFMA_OK;
}

void mlfma_set_destroy(mlfma_set_t s)
{
    if (!s) return;
    {
        DeviceGuard g(s->device);
        if (s->cap) cudaStreamSynchronize(s->cap);
        drop_graphs(s);
        if (s->fork) cudaEventDestroy(s->fork);
        if (s->cap) cudaStreamDestroy(s->cap);
    }
    for (mlfma_plan_t p : s->plans) mlfma_destroy(p);
    delete s;
}

}  // extern "C"
