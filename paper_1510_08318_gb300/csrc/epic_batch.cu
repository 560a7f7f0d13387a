// Batched imaging of many (heterogeneous) sub-arrays: one persistent launch per padded-size
// class, the classes forked onto internal streams and joined back into the caller's stream.
// The EPIC software stacks data streams of several arrays for array operations (App. A.3);
// here the stacking is a list of sub-array segments walked by one kernel.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/epic.h"
#include "epic_internal.h"
#include "epic_plan.h"
#include "epic_trace.h"

namespace {

// Kernel forms a size class can run in: the persistent one-launch form (one CTA, or one cluster
// for N_p >= 256, per image in flight; at N_p = 256 with two row-pass buffers where they fit),
// for N_p = 512 the two-pass form (a row pass and a column pass over every SM, the row-
// transformed grids staged in the class's scratch buffer), and for N_p = 256 the persistent form
// with one row-pass buffer (less shared memory, a cluster barrier per item).
enum ClassForm { kFormPersistent = 0, kFormTwoPass = 1, kFormOneBuffer = 2 };

struct ClassRun {
    int n_pad = 0;
    std::vector<int> members;      // plan indices (at most epic::kMaxSeg)
    cudaStream_t stream = nullptr;
    cudaEvent_t join = nullptr;
    int max_workers = 0;           // 0 = every resident CTA (cluster)
    int form = kFormPersistent;
    float2* scratch = nullptr;     // N_p = 512: the two-pass form's scratch (tp_chunk items)
    int tp_chunk = 0;
};

}  // namespace

struct epic_batch {
    std::vector<epic_plan*> plans;
    std::vector<ClassRun> classes;
    int device = 0, vdt = 0, n_sm = 0;
    bool concurrent = true;        // classes on forked streams (else back to back)
    cudaEvent_t fork = nullptr;
};

namespace {

void destroy_batch(epic_batch* b) {
    if (!b) return;
    for (ClassRun& c : b->classes) {
        if (c.stream) cudaStreamDestroy(c.stream);
        if (c.join) cudaEventDestroy(c.join);
        if (c.scratch) cudaFree(c.scratch);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

epic_status check_call(const epic_batch* b, const void* const* volt, const int* n_time, const float* const* gains,
                       double* const* accum, float* const* image) {
    if (!b) return epic_fail(EPIC_EINVAL, "batch is NULL");
    if (!volt || !n_time || !accum) return epic_fail(EPIC_EINVAL, "NULL argument array");
    for (size_t i = 0; i < b->plans.size(); ++i) {
        if (!volt[i] || !accum[i]) return epic_fail(EPIC_EINVAL, "NULL device array for plan %zu", i);
        const epic_status al = epic_check_alignment({{"volt", volt[i], epic_volt_bytes(b->vdt)},
                                                     {"gains", gains ? gains[i] : nullptr, 8},
                                                     {"accum", accum[i], 8},
                                                     {"image", image ? image[i] : nullptr, 4}});
        if (al != EPIC_OK) {
            const std::string why = epic_last_error();
            return epic_fail(EPIC_EINVAL, "plan %zu: %s", i, why.c_str());
        }
        if (n_time[i] < 1) return epic_fail(EPIC_EINVAL, "n_time[%zu] = %d must be >= 1", i, n_time[i]);
        const long long items = (long long)b->plans[i]->n_chan * b->plans[i]->n_pol * n_time[i];
        if (items > 2147483647LL) return epic_fail(EPIC_EUNSUPPORTED, "plan %zu: C * P * T must stay below 2^31", i);
    }
    for (const ClassRun& c : b->classes) {
        long long tot = 0;
        for (int i : c.members)
            tot += (long long)b->plans[i]->n_chan * b->plans[i]->n_pol * n_time[i];
        if (tot > 2147483647LL) return epic_fail(EPIC_EUNSUPPORTED, "a size class exceeds 2^31 items per call");
    }
    return EPIC_OK;
}

// Enqueue one class on stream st: zero its accumulators, one persistent launch, epilogues.
epic_status run_class(const epic_batch* b, const ClassRun& c, const void* const* volt, const int* n_time,
                      const float* const* gains, double* const* accum, float* const* image, cudaStream_t st,
                      int max_workers, int form) {
    epic::SegList L;
    L.n_seg = (int)c.members.size();
    L.max_ant = 0;
    L.max_workers = max_workers;
    L.max_buffers = form == kFormOneBuffer ? 1 : 0;
    L.first[0] = 0;
    L.cost[0] = 0;
    for (int s = 0; s < L.n_seg; ++s) {
        const int i = c.members[s];
        const epic_plan* p = b->plans[i];
        const int cp = p->n_chan * p->n_pol;
        cudaError_t e = cudaMemsetAsync(accum[i], 0, (size_t)cp * p->n_pad * p->n_pad * sizeof(double), st);
        if (e != cudaSuccess) return epic_cuda_fail(e, "memset accum");
        epic::FwdArgs& a = L.seg[s];
        a = epic_plan_fwd_args(p, volt[i], n_time[i], gains ? reinterpret_cast<const float2*>(gains[i]) : nullptr,
                               accum[i], nullptr);
        L.first[s + 1] = L.first[s] + (int)a.n_items;
        L.weight[s] = epic::item_weight(p->n_pad, p->nnz);
        L.cost[s + 1] = L.cost[s] + L.weight[s] * a.n_items;
        L.max_ant = std::max(L.max_ant, p->n_ant);
    }
    cudaError_t e = form == kFormTwoPass
                        ? epic::launch_fwd512_twopass(b->vdt, L, b->n_sm, st, c.scratch, c.tp_chunk)
                        : epic_launch_fwd_list(c.n_pad, b->vdt, L, b->n_sm, st);
    if (e != cudaSuccess) return epic_cuda_fail(e, "batched imaging kernel launch");
    if (image) {
        for (int i : c.members) {
            if (!image[i]) continue;
            const epic_plan* p = b->plans[i];
            const long long n = (long long)p->n_chan * p->n_pol * p->n_pad * p->n_pad;
            e = epic::launch_finalize_image(accum[i], image[i], n, 1.0 / n_time[i], st);
            if (e != cudaSuccess) return epic_cuda_fail(e, "image epilogue");
        }
    }
    return EPIC_OK;
}

epic_status enqueue(epic_batch* b, const void* const* volt, const int* n_time, const float* const* gains,
                    double* const* accum, float* const* image, cudaStream_t st) {
    if (!b->concurrent) {
        for (const ClassRun& c : b->classes) {
            epic_status s = run_class(b, c, volt, n_time, gains, accum, image, st, c.max_workers, c.form);
            if (s != EPIC_OK) return s;
        }
        return EPIC_OK;
    }
    cudaError_t e = cudaEventRecord(b->fork, st);
    if (e != cudaSuccess) return epic_cuda_fail(e, "fork event");
    // every class stream that waited on the fork is joined back into st, also when a later step
    // fails, so that a stream capture of this call never ends with a stream left unjoined
    epic_status s = EPIC_OK;
    for (ClassRun& c : b->classes) {
        if ((e = cudaStreamWaitEvent(c.stream, b->fork, 0)) != cudaSuccess) {
            s = epic_cuda_fail(e, "fork wait");
            break;
        }
        epic_status r = run_class(b, c, volt, n_time, gains, accum, image, c.stream, c.max_workers, c.form);
        cudaError_t ej = cudaEventRecord(c.join, c.stream);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(st, c.join, 0);
        if (r != EPIC_OK) {
            s = r;
            break;
        }
        if (ej != cudaSuccess) {
            s = epic_cuda_fail(ej, "join");
            break;
        }
    }
    return s;
}

}  // namespace

extern "C" {

epic_status epic_batch_create(epic_batch** batch, int n_plans, epic_plan* const* plans) {
    EpicRange range("epic_batch_create");
    epic_clear_error();
    if (!batch) return epic_fail(EPIC_EINVAL, "batch out-pointer is NULL");
    *batch = nullptr;
    if (n_plans < 1 || !plans) return epic_fail(EPIC_EINVAL, "need at least one plan");
    for (int i = 0; i < n_plans; ++i) {
        if (!plans[i]) return epic_fail(EPIC_EINVAL, "plan %d is NULL", i);
        if (plans[i]->device != plans[0]->device || plans[i]->vdt != plans[0]->vdt)
            return epic_fail(EPIC_EINVAL, "plan %d: all plans of a batch share the device and voltage format", i);
    }
    epic_batch* b = new epic_batch;
    b->plans.assign(plans, plans + n_plans);
    b->device = plans[0]->device;
    b->vdt = plans[0]->vdt;
    b->n_sm = plans[0]->n_sm;
    for (int np : {512, 256, 128, 64, 32}) {
        std::vector<int> m;
        for (int i = 0; i < n_plans; ++i)
            if (plans[i]->n_pad == np) m.push_back(i);
        for (size_t o = 0; o < m.size(); o += epic::kMaxSeg) {
            ClassRun c;
            c.n_pad = np;
            c.members.assign(m.begin() + o, m.begin() + std::min(m.size(), o + (size_t)epic::kMaxSeg));
            b->classes.push_back(c);
        }
    }
    EpicDeviceGuard guard(b->device);
    cudaError_t e = guard.ok ? cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) : cudaErrorInvalidDevice;
    for (ClassRun& c : b->classes) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.join, cudaEventDisableTiming);
        // the two-pass form's scratch, so that the autotuner can choose it and a call allocates
        // nothing (each N_p = 512 class its own: classes may run concurrently)
        if (e == cudaSuccess && c.n_pad == 512) {
            int max_ant = 0;
            for (int i : c.members) max_ant = std::max(max_ant, plans[i]->n_ant);
            int smem_optin = 0;
            cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
            if (epic::twopass_rows_smem_bytes(max_ant) <= (size_t)smem_optin) {
                c.tp_chunk = 4 * b->n_sm;
                e = cudaMalloc(reinterpret_cast<void**>(&c.scratch), epic::twopass_scratch_bytes(c.tp_chunk));
                if (e != cudaSuccess) c.scratch = nullptr;
            }
        }
    }
    if (e != cudaSuccess) {
        destroy_batch(b);
        return epic_cuda_fail(e, "batch streams");
    }
    *batch = b;
    return EPIC_OK;
}

void epic_batch_destroy(epic_batch* batch) {
    if (!batch) return;
    EpicDeviceGuard guard(batch->device);
    destroy_batch(batch);
}

epic_status epic_batch_image(epic_batch* batch, const void* const* volt, const int* n_time, const float* const* gains,
                             double* const* accum, float* const* image, void* stream) {
    EpicRange range("epic_batch_image");
    epic_clear_error();
    epic_status s = check_call(batch, volt, n_time, gains, accum, image);
    if (s != EPIC_OK) return s;
    EpicDeviceGuard guard(batch->device);
    if (!guard.ok) return epic_fail(EPIC_ECUDA, "cannot select CUDA device %d", batch->device);
    return enqueue(batch, volt, n_time, gains, accum, image, static_cast<cudaStream_t>(stream));
}

epic_status epic_batch_autotune(epic_batch* batch, const void* const* volt, const int* n_time,
                                const float* const* gains, double* const* accum, void* stream) {
    EpicRange range("epic_batch_autotune");
    epic_clear_error();
    epic_status s = check_call(batch, volt, n_time, gains, accum, nullptr);
    if (s != EPIC_OK) return s;
    EpicDeviceGuard guard(batch->device);
    if (!guard.ok) return epic_fail(EPIC_ECUDA, "cannot select CUDA device %d", batch->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // timing events, destroyed on every way out of this call
    struct Events {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ~Events() {
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
        }
    } ev;
    cudaError_t e = cudaEventCreate(&ev.e0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev.e1);
    if (e != cudaSuccess) return epic_cuda_fail(e, "autotune events");
    cudaEvent_t e0 = ev.e0, e1 = ev.e1;
    auto time_it = [&](auto&& body, float& ms) -> epic_status {
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, st);
            epic_status r = body();
            if (r != EPIC_OK) return r;
            cudaEventRecord(e1, st);
            cudaError_t err = cudaEventSynchronize(e1);
            if (err != cudaSuccess) return epic_cuda_fail(err, "autotune run");
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            best = std::min(best, t);
        }
        ms = best;
        return EPIC_OK;
    };
    // 1) per class: the kernel form and worker count that run it fastest alone -- the persistent
    //    form with all, 3/4 or 1/2 of its resident CTAs (clusters), for N_p = 512 also the
    //    two-pass form on every SM, for N_p = 256 also the one-buffer form at the best count
    std::vector<float> alone(batch->classes.size(), 0.f);
    for (size_t k = 0; k < batch->classes.size() && s == EPIC_OK; ++k) {
        ClassRun& c = batch->classes[k];
        const int full = epic_resident_workers(c.n_pad, batch->vdt, batch->plans, c.members, batch->n_sm);
        int best_w = 0, best_f = kFormPersistent;
        float best_t = 1e30f;
        for (int frac4 : {4, 3, 2}) {
            const int w = frac4 == 4 ? 0 : std::max(1, full * frac4 / 4);
            float t = 0.f;
            s = time_it([&] { return run_class(batch, c, volt, n_time, gains, accum, nullptr, st, w, kFormPersistent); },
                        t);
            if (s != EPIC_OK) break;
            if (t < best_t) {
                best_t = t;
                best_w = w;
            }
        }
        if (s == EPIC_OK && c.scratch) {
            float t = 0.f;
            s = time_it([&] { return run_class(batch, c, volt, n_time, gains, accum, nullptr, st, 0, kFormTwoPass); }, t);
            if (s == EPIC_OK && t < best_t) {
                best_t = t;
                best_w = 0;
                best_f = kFormTwoPass;
            }
        }
        if (s == EPIC_OK && c.n_pad == 256) {
            float t = 0.f;
            s = time_it([&] { return run_class(batch, c, volt, n_time, gains, accum, nullptr, st, best_w, kFormOneBuffer); },
                        t);
            if (s == EPIC_OK && t < best_t) {
                best_t = t;
                best_f = kFormOneBuffer;
            }
        }
        c.max_workers = best_w;
        c.form = best_f;
        alone[k] = best_t;
    }
    // 2) classes back to back vs concurrently (forked streams), timed alternately (twice the
    //    best of three each, so that drifting clocks or a busy neighbour affect both alike).  Timed eagerly, the
    //    concurrent schedule also pays one stream fork and join per class, which a captured graph
    //    replays without host work; it is kept unless back to back is faster by more than that
    //    allowance (2 %).
    if (s == EPIC_OK && batch->classes.size() > 1) {
        float t_seq = 1e30f, t_con = 1e30f;
        for (int rep = 0; rep < 2 && s == EPIC_OK; ++rep) {
            for (int con = 0; con < 2 && s == EPIC_OK; ++con) {
                batch->concurrent = con != 0;
                float t = 0.f;
                s = time_it([&] { return enqueue(batch, volt, n_time, gains, accum, nullptr, st); }, t);
                float& best = con ? t_con : t_seq;
                best = std::min(best, t);
            }
        }
        if (s == EPIC_OK) batch->concurrent = t_seq >= 0.98f * t_con;
    }
    return s;
}

epic_status epic_batch_class(const epic_batch* batch, int k, int* n_pad, int* workers, int* form) {
    epic_clear_error();
    if (!batch) return epic_fail(EPIC_EINVAL, "batch is NULL");
    if (k < 0 || k >= (int)batch->classes.size())
        return epic_fail(EPIC_EINVAL, "class %d of %d", k, (int)batch->classes.size());
    const ClassRun& c = batch->classes[k];
    if (n_pad) *n_pad = c.n_pad;
    if (workers) *workers = c.max_workers;
    if (form) *form = c.form;
    return EPIC_OK;
}

epic_status epic_batch_info(const epic_batch* batch, int* n_classes, int* concurrent, int* workers, int max_workers) {
    epic_clear_error();
    if (!batch) return epic_fail(EPIC_EINVAL, "batch is NULL");
    if (n_classes) *n_classes = (int)batch->classes.size();
    if (concurrent) *concurrent = batch->concurrent ? 1 : 0;
    if (workers)
        for (int k = 0; k < (int)batch->classes.size() && k < max_workers; ++k) workers[k] = batch->classes[k].max_workers;
    return EPIC_OK;
}

}  // extern "C"
