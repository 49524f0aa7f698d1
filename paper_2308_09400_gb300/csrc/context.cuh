// Context: the device it is bound to and the scratch buffers it owns (internal).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

#include "common.cuh"

// A growable device buffer owned by a context.
struct gipc_scratch {
    void* ptr = nullptr;
    size_t bytes = 0;
    // Ensure at least `want` bytes; reallocates (contents lost) when growing.
    gipc_status reserve(size_t want) {
        if (want <= bytes) return GIPC_OK;
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
        size_t sz = want + want / 4 + 256;
        if (cudaMalloc(&ptr, sz) != cudaSuccess) {
            cudaGetLastError();
            return gipc::fail(GIPC_ERR_OOM, "device scratch allocation of %zu bytes failed", sz);
        }
        bytes = sz;
        return GIPC_OK;
    }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
    template <typename T>
    T* as() const { return static_cast<T*>(ptr); }
};

// Per-kernel timing with CUDA events recorded on the launching stream (enabled on demand).
struct gipc_profiler {
    static constexpr int kKinds = GIPC_PROF_KINDS;
    bool on = false;
    std::vector<cudaEvent_t> pool[kKinds];
    int used[kKinds] = {};
    int every[kKinds] = {};       // record one launch in `every` (0 or 1: all)
    unsigned seen[kKinds] = {};   // launches of the kind since profiling began
    bool open[kKinds] = {};       // the current launch is being recorded
    cudaEvent_t take(int kind) {
        if (used[kind] == (int)pool[kind].size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pool[kind].push_back(e);
        }
        return pool[kind][used[kind]++];
    }
    // record a start / stop pair around one launch of `kind` (a sampled subset, if so set)
    void start(int kind, cudaStream_t s) {
        if (!on) return;
        open[kind] = every[kind] <= 1 || seen[kind] % (unsigned)every[kind] == 0;
        ++seen[kind];
        if (open[kind]) record(kind, s);
    }
    void stop(int kind, cudaStream_t s) {
        if (on && open[kind]) record(kind, s);
        open[kind] = false;
    }
    void record(int kind, cudaStream_t s) {
        cudaEvent_t e = take(kind);
        if (e) cudaEventRecord(e, s);
    }
    void reset() {
        for (int k = 0; k < kKinds; ++k) {
            used[k] = 0;
            seen[k] = 0;
            open[k] = false;
        }
    }
    void release() {
        for (auto& v : pool)
            for (auto e : v) cudaEventDestroy(e);
        for (auto& v : pool) v.clear();
        reset();
    }
};

// Records one span of `kind` around a scope (no-op while profiling is off).
struct gipc_prof_span {
    gipc_profiler& p;
    int kind;
    cudaStream_t s;
    gipc_prof_span(gipc_profiler& p_, int k, cudaStream_t s_) : p(p_), kind(k), s(s_) { p.start(kind, s); }
    ~gipc_prof_span() { p.stop(kind, s); }
};

// Candidate pairs of the contact broad phase kept between the detections of one time step: built
// with boxes padded by dhat + 2 margin around the positions x_b, they contain every pair closer
// than dhat at any x with max |x - x_b| <= margin (per axis), and every pair whose swept boxes
// overlap for a step d with 2 (max |x - x_b| + max |d|) <= dhat + 2 margin.
struct gipc_contact_cache {
    bool valid = false;
    int64_t n = 0, npt = 0, np = 0;          // vertex count, point-triangle pairs, all pairs
    const int32_t *tris = nullptr, *edges = nullptr, *verts = nullptr;
    int64_t ntri = 0, nedge = 0, nvert = 0;
    const int32_t* vscene = nullptr;         // batched scenes: the vertex -> scene map, and their count
    int nscenes = 1;
    double dhat = 0.0, margin = 0.0, pad = 0.0;

    // Margin tuner.  A wider margin means fewer rebuilds but more candidates to classify and test,
    // and which wins depends on the scene.  The detections between two builds form an epoch; its
    // GPU time (detections and cached CCD steps, CUDA events on the stream) per detection is
    // credited to the margin level it was built with.  A build picks the level with the lowest
    // time per detection so far, after trying the next wider level once when the surface outran
    // the margin.  Levels are kMargin[l] dhat.  The choice changes timing only: the contact sets
    // and steps are those of a fresh broad phase whatever the margin.
    static constexpr int kLevels = 4;
    static constexpr double kMargin[kLevels] = {0.5, 1.0, 2.0, 4.0};
    int level = 0;                                // level of the next build
    int built = 0;                                // level of the current candidates
    double cost[kLevels] = {}, dets[kLevels] = {};   // decayed GPU ms and detections per level
    double epoch_ms = 0.0;
    int epoch_dets = 0;
    double tuned_dhat = -1.0;                     // scene key of the statistics (dhat, batched)
    bool tuned_batch = false;
    cudaEvent_t ev[2][2] = {};                    // [detection, CCD][start, stop]
    bool pending[2] = {};
    void release_events() {
        for (auto& k : ev)
            for (auto& e : k) {
                if (e) cudaEventDestroy(e);
                e = nullptr;
            }
        pending[0] = pending[1] = false;
    }
};

// Run-time choice of the batched product's staging variant for one (precision, size class).
struct gipc_spmv_tune {
    int prec = 0, size_class = 0, chosen = -1;
    double sum_ms[GIPC_SPMV_VARIANTS] = {};
    int cnt[GIPC_SPMV_VARIANTS] = {};
};


struct gipc_ctx {
    int device = 0;
    static constexpr int kSlots = 66;   // assembly 0-8 and 61, pcg 9-15, 40, 62 and 65, contacts 16-19, 30-39, 45-46, 59-60 and 63-64, time step 20-29, 41-44 and 47-48, derivatives 49-58
    gipc_scratch slot[kSlots];
    gipc_profiler prof;
    gipc_contact_cache ccache;   // filled and used by the time step only
    bool solver_trace = false;   // persistent solves record phase stamps (gipc_profile_solver_trace)
    int solver_trace_iters = 0;  // iterations of the last traced solve
    bool spmv_autotune = true;   // batched product variant chosen at run time (gipc_spmv_autotune)
    bool batch_loop = true;      // batched solves as one persistent launch (gipc_pcg_batch_persistent)
    std::vector<gipc_spmv_tune> spmv_tunes;
    cudaEvent_t spmv_ev[2] = {nullptr, nullptr};   // around one timed chunk of iterations
    void release_all() {
        for (auto& s : slot) s.release();
        prof.release();
        ccache.valid = false;
        ccache.release_events();
        for (auto& e : spmv_ev) {
            if (e) cudaEventDestroy(e);
            e = nullptr;
        }
    }
};
