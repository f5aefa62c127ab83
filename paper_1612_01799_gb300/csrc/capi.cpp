// C-ABI of the solver (include/poisson.h): plan creation (setup phase), solves, facts.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/poisson.h"
#include "setup.h"
#include "solver.h"

namespace gsp {
// Per arithmetic (FP32, FP64, double-float) entry points of the pass code.
#define GSP_ARITH_DECL(sfx)                                                                                        \
    cudaError_t solve_##sfx(const DevicePlan &, const PtrArray &, const PtrArray &, int, cudaStream_t, cudaEvent_t *, \
                            double *, int);                                                                        \
    cudaError_t xy_slab_##sfx(const DevicePlan &, const void *, void *, int, int, cudaStream_t, bool);            \
    cudaError_t symbol_table_##sfx(const DevicePlan &, const double *, const double *, int, double, double, double, \
                                   int, cudaStream_t);                                                             \
    cudaError_t symbol_table_box_##sfx(const DevicePlan &, const double *, const double *, int, double, double,    \
                                       double, const double *, int, cudaStream_t);                                 \
    cudaError_t encode_maps_##sfx(DevicePlan &);                                                                   \
    cudaError_t z_pass_##sfx(const DevicePlan &, cudaStream_t);                                                    \
    cudaError_t z_lines_##sfx(const DevicePlan &, int, int, cudaStream_t);                                         \
    cudaError_t y_passes_##sfx(const DevicePlan &, cudaStream_t);                                                  \
    cudaError_t x_passes_##sfx(const DevicePlan &, cudaStream_t);                                                  \
    cudaError_t xy_passes_##sfx(const DevicePlan &, cudaStream_t);
GSP_ARITH_DECL(f32)
GSP_ARITH_DECL(f64)
GSP_ARITH_DECL(df)
#undef GSP_ARITH_DECL

// The entry point of `name` for p's arithmetic.
#define GSP_BY_ARITH(p, name, ...)                                                                 \
    ((p).dtype == POISSON_F32 ? name##_f32(__VA_ARGS__)                                            \
                              : (p).arith ? name##_df(__VA_ARGS__) : name##_f64(__VA_ARGS__))

cudaError_t launch_xy_slab(const DevicePlan &p, const void *rho, void *u, int z0, int nz, cudaStream_t s, bool fwd) {
    return GSP_BY_ARITH(p, xy_slab, p, rho, u, z0, nz, s, fwd);
}
cudaError_t launch_xy_passes(const DevicePlan &p, cudaStream_t s) { return GSP_BY_ARITH(p, xy_passes, p, s); }
cudaError_t launch_x_passes(const DevicePlan &p, cudaStream_t s) { return GSP_BY_ARITH(p, x_passes, p, s); }
cudaError_t launch_y_passes(const DevicePlan &p, cudaStream_t s) { return GSP_BY_ARITH(p, y_passes, p, s); }
cudaError_t launch_z_pass(const DevicePlan &p, cudaStream_t s) { return GSP_BY_ARITH(p, z_pass, p, s); }
cudaError_t encode_tma_maps(DevicePlan &p) { return GSP_BY_ARITH(p, encode_maps, p); }

static const int kSupportedN[] = {4, 8, 16, 32, 48, 64, 80, 96, 128, 160, 192, 256, 320, 384, 512, 1024};

bool n_supported(int N) {
    for (int n : kSupportedN)
        if (n == N) return true;
    return false;
}

bool n_any(int N) {
    if (N < 4 || N > 1024 || (N & 1)) return false;
    for (int f : {2, 3, 5})
        while (N % f == 0) N /= f;
    return N == 1;
}

AnySched any_sched(int L) {
    AnySched s{};
    s.L = L;
    int m = L, n = 0;
    for (int f : {5, 3})
        while (m % f == 0 && n < kAnyMaxStages) {
            s.r[n++] = f;
            m /= f;
        }
    while (m % 4 == 0 && n < kAnyMaxStages) {
        s.r[n++] = 4;
        m /= 4;
    }
    if (m == 2 && n < kAnyMaxStages) {
        s.r[n++] = 2;
        m = 1;
    }
    s.nst = m == 1 ? n : 0;
    unsigned long long ns = 1;
    for (int st = 0; st < s.nst; ++st) {
        s.mul[st] = ns == 1 ? 0u : (unsigned)((1ull << 32) / ns + 1);
        ns *= (unsigned long long)s.r[st];
    }
    return s;
}

cudaError_t launch_solve(const DevicePlan &p, const PtrArray &rho, const PtrArray &u, int count,
                         cudaStream_t s, cudaEvent_t *ev, double *tail, int skip) {
    if (count < 1 || count > p.max_batch || count > kMaxBatch) return cudaErrorInvalidValue;
    return GSP_BY_ARITH(p, solve, p, rho, u, count, s, ev, tail, skip);
}

// Streams that poisson_solve_batched forks independent plan groups onto (per device,
// created with the first plan on the device, so that a batched call can be captured).
struct ForkPool {
    static constexpr int kStreams = 8;
    bool ready = false;
    cudaStream_t st[kStreams];
    cudaEvent_t fork, join[kStreams];
};
static ForkPool g_pools[64];
static std::mutex g_pool_mutex;

static cudaError_t fork_pool(int dev, ForkPool **out) {
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    ForkPool &fp = g_pools[dev];
    if (!fp.ready) {
        cudaError_t e;
        for (int i = 0; i < ForkPool::kStreams; ++i) {
            if ((e = cudaStreamCreateWithFlags(&fp.st[i], cudaStreamNonBlocking)) != cudaSuccess) return e;
            if ((e = cudaEventCreateWithFlags(&fp.join[i], cudaEventDisableTiming)) != cudaSuccess) return e;
        }
        if ((e = cudaEventCreateWithFlags(&fp.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
        fp.ready = true;
    }
    *out = &fp;
    return cudaSuccess;
}

cudaError_t launch_symbol_table_box(const DevicePlan &p, const double *dA3, const double *dw, int nterms,
                                    double C0, double C2, double scale, const double *l, int literal,
                                    cudaStream_t s) {
    return GSP_BY_ARITH(p, symbol_table_box, p, dA3, dw, nterms, C0, C2, scale, l, literal, s);
}
cudaError_t launch_symbol_table(const DevicePlan &p, const double *dA, const double *dw,
                                int nterms, double C0, double C2, double scale, int literal,
                                cudaStream_t s) {
    return GSP_BY_ARITH(p, symbol_table, p, dA, dw, nterms, C0, C2, scale, literal, s);
}

// ---- autotuning of kernel variants --------------------------------------------------------
// Decisions per (device, N, dtype), made by the first plan of that shape and reused.  With
// the environment variable POISSON_TUNE_CACHE naming a file, decisions also persist across
// processes: the file is read once, and each new decision is appended to it.  Lines are
//   <N> <dtype> <zform> <yform> <xform> <xyform> <arith> <device name>
// after a first line "gspoisson-tune 1"; a decision read from the file applies to every
// device of that name, and lines that do not parse, or name a form that does not exist
// for their shape, are ignored.
struct TuneEntry {
    int dev, N, dtype, zform, yform, xform, xyform, arith;
};
static std::vector<TuneEntry> g_tune;
static std::mutex g_tune_mutex;

struct FileTune {
    std::string name;
    int N, dtype, zform, yform, xform, xyform, arith;
};
static std::vector<FileTune> g_file_tune;
static bool g_file_tune_read = false;
static const char *kTuneHeader = "gspoisson-tune 1";

static std::string device_name(int dev) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return std::string();
    return std::string(prop.name);
}

static bool forms_valid(int N, int dtype, int arith, int zf, int yf, int xf, int xyf) {
    return zf >= 0 && zf < 3 && (z_forms(N, dtype, arith) >> zf & 1) && yf >= 0 && yf < 2 &&
           (y_forms(N, dtype) >> yf & 1) && xf >= 0 && xf < 2 && (x_forms(N, dtype) >> xf & 1) &&
           xyf >= 0 && xyf < 2 && (xy_forms(N, dtype) >> xyf & 1);
}

// Called with g_tune_mutex held.
static void read_tune_file() {
    if (g_file_tune_read) return;
    g_file_tune_read = true;
    const char *path = std::getenv("POISSON_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char line[512];
    bool header = false;
    while (std::fgets(line, sizeof line, f)) {
        line[strcspn(line, "\r\n")] = 0;
        if (!header) {
            header = std::strcmp(line, kTuneHeader) == 0;
            if (!header) break;
            continue;
        }
        FileTune t;
        int used = 0;
        if (std::sscanf(line, "%d %d %d %d %d %d %d %n", &t.N, &t.dtype, &t.zform, &t.yform, &t.xform, &t.xyform,
                        &t.arith, &used) != 7 ||
            used <= 0 || !line[used])
            continue;
        t.name = line + used;
        if (!n_supported(t.N) || (t.dtype != POISSON_F32 && t.dtype != POISSON_F64)) continue;
        if (t.arith != 0 && (t.arith != 1 || t.dtype != POISSON_F64)) continue;
        if (!forms_valid(t.N, t.dtype, t.arith, t.zform, t.yform, t.xform, t.xyform)) continue;
        g_file_tune.push_back(t);
    }
    std::fclose(f);
}

// Called with g_tune_mutex held.
static void append_tune_file(const TuneEntry &t, const std::string &name) {
    const char *path = std::getenv("POISSON_TUNE_CACHE");
    if (!path || !*path || name.empty()) return;
    FILE *f = std::fopen(path, "r");
    bool fresh = true;
    if (f) {
        fresh = std::fgetc(f) == EOF;
        std::fclose(f);
    }
    f = std::fopen(path, "a");
    if (!f) return;
    if (fresh) std::fprintf(f, "%s\n", kTuneHeader);
    std::fprintf(f, "%d %d %d %d %d %d %d %s\n", t.N, t.dtype, t.zform, t.yform, t.xform, t.xyform, t.arith,
                 name.c_str());
    std::fclose(f);
}

// A decision for p's shape on device dev, from this process or the cache file: true and
// p's forms set, or false.  Called with g_tune_mutex held.
static bool lookup_tune(DevicePlan &p, int dev) {
    for (const TuneEntry &t : g_tune)
        if (t.dev == dev && t.N == p.N && t.dtype == p.dtype) {
            p.zform = t.zform;
            p.yform = t.yform;
            p.xform = t.xform;
            p.xyform = t.xyform;
            p.arith = t.arith;
            return true;
        }
    read_tune_file();
    if (g_file_tune.empty()) return false;
    const std::string name = device_name(dev);
    for (const FileTune &t : g_file_tune)
        if (t.N == p.N && t.dtype == p.dtype && t.name == name) {
            // A plan without the counter block cannot run the fused x-y form.
            const int xyf = p.sync ? t.xyform : 0;
            g_tune.push_back(TuneEntry{dev, p.N, p.dtype, t.zform, t.yform, t.xform, t.xyform, t.arith});
            p.zform = t.zform;
            p.yform = t.yform;
            p.xform = t.xform;
            p.xyform = xyf;
            p.arith = t.arith;
            return true;
        }
    return false;
}

// Mean time (ms) of `reps` runs of `run` (one density) after one warm-up run.
template <class Run>
static cudaError_t time_runs(Run &&run, cudaStream_t s, cudaEvent_t a, cudaEvent_t b, int reps, float *ms) {
    cudaError_t e;
    if ((e = run()) != cudaSuccess) return e;
    if ((e = cudaEventRecord(a, s)) != cudaSuccess) return e;
    for (int i = 0; i < reps; ++i)
        if ((e = run()) != cudaSuccess) return e;
    if ((e = cudaEventRecord(b, s)) != cudaSuccess) return e;
    if ((e = cudaEventSynchronize(b)) != cudaSuccess) return e;
    if ((e = cudaEventElapsedTime(ms, a, b)) != cudaSuccess) return e;
    *ms /= reps;
    return cudaSuccess;
}

// Index of the fastest set bit of `forms` (form v timed with *field = v), or an error.
template <class Run>
static cudaError_t pick_form(int forms, int *field, Run &&run, cudaStream_t s, cudaEvent_t a, cudaEvent_t b) {
    int best = 0;
    float best_ms = 0.f;
    for (int v = 0; v < 3; ++v) {
        if (!(forms >> v & 1)) continue;
        float ms = 0.f;
        *field = v;
        cudaError_t e = time_runs(run, s, a, b, 3, &ms);
        if (e != cudaSuccess) {
            *field = 0;
            return e;
        }
        if (v == 0 || ms < best_ms) {
            best = v;
            best_ms = ms;
        }
    }
    *field = best;
    return cudaSuccess;
}

// Choose p.arith (FP64 plans), p.zform, p.yform, p.xform and p.xyform: the cached decision
// for this shape, else the fastest forms that exist, timed on p's zeroed workspace.  An FP64
// plan first times its passes (block forms) in FP64 and in double-float arithmetic and keeps
// the faster; timing needs no valid tables, so the caller builds the twiddles and the symbol
// afterwards, in the chosen arithmetic's format.  The z pass writes only w3, the y passes w2
// and w1, the x passes (timed with w2 as density and output) w1 and w2, the x-y passes all
// three, and every solve writes each of them before reading it.  The x-y form is timed last,
// against the separate passes in the y and x forms just chosen.
static cudaError_t autotune(DevicePlan &p, int dev) {
    p.zform = 0;
    p.yform = 0;
    p.xform = 0;
    p.xyform = 0;
    p.arith = 0;
    // The runtime-length forms have one form per pass; only an FP64 plan's arithmetic is
    // timed, and (their shapes being many) the choice is not cached.
    const bool any = p.any != 0;
    const int zf = any ? 1 : z_forms(p.N, p.dtype), yf = any ? 1 : y_forms(p.N, p.dtype);
    const int xf = any ? 1 : x_forms(p.N, p.dtype);
    const int xyf = p.sync && !any ? xy_forms(p.N, p.dtype) : 1;
    const int af = p.dtype == POISSON_F64 ? 3 : 1;
    if (zf == 1 && yf == 1 && xf == 1 && xyf == 1 && af == 1) return cudaSuccess;
    if (!any) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        if (lookup_tune(p, dev)) return cudaSuccess;
    }
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess && af != 1)
        e = pick_form(af, &p.arith, [&] {
            cudaError_t r = launch_x_passes(p, s);
            if (r == cudaSuccess) r = launch_y_passes(p, s);
            return r == cudaSuccess ? launch_z_pass(p, s) : r;
        }, s, a, b);
    if (e == cudaSuccess)
        e = pick_form(any ? 1 : z_forms(p.N, p.dtype, p.arith), &p.zform, [&] { return launch_z_pass(p, s); }, s, a,
                      b);
    if (e == cudaSuccess) e = pick_form(yf, &p.yform, [&] { return launch_y_passes(p, s); }, s, a, b);
    if (e == cudaSuccess) e = pick_form(xf, &p.xform, [&] { return launch_x_passes(p, s); }, s, a, b);
    if (e == cudaSuccess) e = pick_form(xyf, &p.xyform, [&] { return launch_xy_passes(p, s); }, s, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        p.zform = p.yform = p.xform = p.xyform = p.arith = 0;
        return e;
    }
    if (any) return cudaSuccess;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    for (const TuneEntry &t : g_tune)  // another thread may have decided meanwhile
        if (t.dev == dev && t.N == p.N && t.dtype == p.dtype) {
            p.zform = t.zform;
            p.yform = t.yform;
            p.xform = t.xform;
            p.xyform = t.xyform;
            p.arith = t.arith;
            return cudaSuccess;
        }
    const TuneEntry mine{dev, p.N, p.dtype, p.zform, p.yform, p.xform, p.xyform, p.arith};
    g_tune.push_back(mine);
    append_tune_file(mine, device_name(dev));
    return cudaSuccess;
}
}  // namespace gsp

struct poisson_plan_s {
    gsp::HostTables ht;
    gsp::DevicePlan dp;
    int device = 0;
    int correction = 0;      // POISSON_KNOB_CORRECTION: 0 fused, 1 the unpadded transform pair
    size_t elem = 0;         // bytes per real value
    size_t ws_bytes = 0;
    size_t table_bytes = 0;
    void *stage_in = nullptr;   // device staging for poisson_solve_host
    void *stage_out = nullptr;
    cudaEvent_t ev[6] = {};
    bool have_events = false;
    // poisson_solve_host's slab pipeline: a copy stream and one event per slab and
    // direction, made on first use.
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t slab_ev[2 * 8 + 1] = {};
    bool have_slab_events = false;
};

namespace gsp {
static thread_local cudaError_t t_last_error = cudaSuccess;
void note_cuda_error(cudaError_t e) {
    if (e != cudaSuccess) t_last_error = e;
}
}  // namespace gsp

extern "C" const char *poisson_last_cuda_error(void) {
    return gsp::t_last_error == cudaSuccess ? "none" : cudaGetErrorName(gsp::t_last_error);
}

static int map_cuda(cudaError_t e) {
    gsp::note_cuda_error(e);
    if (e == cudaSuccess) return POISSON_OK;
    if (e == cudaErrorMemoryAllocation) return POISSON_ERR_ALLOC;
    return POISSON_ERR_CUDA;
}

static void free_plan(poisson_plan p) {
    if (!p) return;
    void *twc = p->dp.twc != p->dp.tw ? p->dp.twc : nullptr;
    void *bufs[] = {p->dp.sym, p->dp.symT, p->dp.tw, twc, p->dp.w1, p->dp.w2, p->dp.w3, p->dp.status,
                    p->dp.tail, p->dp.sync, p->stage_in, p->stage_out};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (p->have_events)
        for (auto &e : p->ev) cudaEventDestroy(e);
    if (p->have_slab_events)
        for (auto &e : p->slab_ev) cudaEventDestroy(e);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    delete p;
}

extern "C" int poisson_supported_n(int N) { return gsp::n_supported(N) ? 1 : gsp::n_any(N) ? 2 : 0; }

extern "C" const char *poisson_strerror(int code) {
    switch (code) {
        case POISSON_OK: return "ok";
        case POISSON_ERR_ARG: return "invalid argument";
        case POISSON_ERR_ALLOC: return "allocation failed";
        case POISSON_ERR_CUDA: return "CUDA error";
        case POISSON_ERR_UNSUPPORTED: return "unsupported size";
        case POISSON_ERR_TIMEOUT: return "device wait timed out";
        case POISSON_ERR_NUMERIC: return "requested accuracy not reachable";
        default: return "unknown error";
    }
}

extern "C" int poisson_plan_create(poisson_plan *out, int N, double L, double tol, int dtype) {
    return poisson_plan_create_batched(out, N, L, tol, dtype, 1);
}

static int plan_create_impl(poisson_plan *out, const int *n3, double L, const double *L3, double tol, int dtype,
                            int max_batch);

extern "C" int poisson_plan_create_batched(poisson_plan *out, int N, double L, double tol, int dtype,
                                           int max_batch) {
    const int n3[3] = {N, N, N};
    return plan_create_impl(out, n3, L, nullptr, tol, dtype, max_batch);
}

extern "C" int poisson_plan_create_box(poisson_plan *out, int N, double Lx, double Ly, double Lz, double tol,
                                       int dtype) {
    const int n3[3] = {N, N, N};
    const double L3[3] = {Lx, Ly, Lz};
    return plan_create_impl(out, n3, 0.0, L3, tol, dtype, 1);
}

extern "C" int poisson_plan_create_box_n(poisson_plan *out, int nx, int ny, int nz, double Lx, double Ly, double Lz,
                                         double tol, int dtype) {
    const int n3[3] = {nx, ny, nz};
    const double L3[3] = {Lx, Ly, Lz};
    return plan_create_impl(out, n3, 0.0, L3, tol, dtype, 1);
}

// Twiddles W_{2N}^e from FP64 (long double arithmetic) into the plan's tables, in its
// arithmetic's format: FP32 rounded once (and the column passes' (re, re, im, im) copy), FP64,
// or double-float (re.hi, re.lo, im.hi, im.lo) split from the FP64 value.
static cudaError_t upload_table(void *dst, int n2, int dtype, int arith) {
    std::vector<double> tw;
    gsp::twiddles(n2, tw);
    const size_t n = (size_t)n2;
    if (dtype == POISSON_F32) {
        std::vector<float> twf(tw.begin(), tw.end());
        return cudaMemcpy(dst, twf.data(), n * 2 * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (!arith) return cudaMemcpy(dst, tw.data(), n * 2 * sizeof(double), cudaMemcpyHostToDevice);
    std::vector<float> twd(n * 4);
    for (size_t i = 0; i < 2 * n; ++i) {
        const float hi = (float)tw[i];
        twd[2 * i] = hi;
        twd[2 * i + 1] = (float)(tw[i] - (double)hi);
    }
    return cudaMemcpy(dst, twd.data(), n * 4 * sizeof(float), cudaMemcpyHostToDevice);
}

static cudaError_t upload_twiddles(poisson_plan p) {
    if (p->dp.any) {
        // W_{2 n_q}^e of each axis, in the arithmetic's storage.
        for (int q = 0; q < 3; ++q) {
            cudaError_t e = upload_table(p->dp.tw3[q], 2 * p->dp.n3[q], p->dp.dtype, p->dp.arith);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const int N = p->dp.N;
    std::vector<double> tw;
    gsp::twiddles(2 * N, tw);
    const size_t n = (size_t)2 * N;
    cudaError_t e;
    if (p->dp.dtype == POISSON_F32) {
        std::vector<float> twf(tw.begin(), tw.end());
        e = cudaMemcpy(p->dp.tw, twf.data(), n * 2 * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
        std::vector<float> tw4(n * 4);
        for (size_t i = 0; i < n; ++i) {
            tw4[4 * i] = tw4[4 * i + 1] = (float)tw[2 * i];
            tw4[4 * i + 2] = tw4[4 * i + 3] = (float)tw[2 * i + 1];
        }
        return cudaMemcpy(p->dp.twc, tw4.data(), n * 4 * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (!p->dp.arith) return cudaMemcpy(p->dp.tw, tw.data(), n * 2 * sizeof(double), cudaMemcpyHostToDevice);
    std::vector<float> twd(n * 4);
    for (size_t i = 0; i < 2 * n; ++i) {
        const float hi = (float)tw[i];
        twd[2 * i] = hi;
        twd[2 * i + 1] = (float)(tw[i] - (double)hi);
    }
    return cudaMemcpy(p->dp.tw, twd.data(), n * 4 * sizeof(float), cudaMemcpyHostToDevice);
}

static int plan_create_impl(poisson_plan *out, const int *n3, double L, const double *L3, double tol, int dtype,
                            int max_batch) {
    if (!out) return POISSON_ERR_ARG;
    *out = nullptr;
    if (dtype != POISSON_F32 && dtype != POISSON_F64) return POISSON_ERR_ARG;
    for (int q = 0; q < 3; ++q)
        if (n3[q] < 4 || n3[q] > 1024 || (n3[q] & 1)) return POISSON_ERR_ARG;
    if (max_batch < 1 || max_batch > gsp::kMaxBatch) return POISSON_ERR_ARG;
    const int N = n3[0];
    const bool cube_n = n3[1] == N && n3[2] == N;
    // The compiled-length forms serve the sizes they were built for, the same on every axis;
    // every other even 5-smooth count (and any mix of them) runs the runtime-length forms.
    const bool any = !(cube_n && gsp::n_supported(N));
    if (any && !(gsp::n_any(n3[0]) && gsp::n_any(n3[1]) && gsp::n_any(n3[2]))) return POISSON_ERR_UNSUPPORTED;
    if (any && L3 && max_batch != 1) return POISSON_ERR_ARG;
    poisson_plan p = new (std::nothrow) poisson_plan_s();
    if (!p) return POISSON_ERR_ALLOC;
    // The Gaussian sum, delta, eps and the near-zone constants on the host; the per-axis
    // table A_j(k) below on the device.
    int rc = L3 ? gsp::build_host_scalars_box(n3, L3, tol, p->ht) : gsp::build_host_scalars(N, L, tol, p->ht);
    if (rc != POISSON_OK) {
        delete p;
        return rc;
    }
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return map_cuda(e);
    }
    const int nx = n3[0], ny = n3[1], nz = n3[2];
    p->elem = dtype == POISSON_F32 ? 4 : 8;
    p->dp.max_batch = max_batch;
    p->dp.N = N;
    p->dp.dtype = dtype;
    p->dp.any = any ? 1 : 0;
    for (int q = 0; q < 3; ++q) p->dp.n3[q] = n3[q];
    p->dp.Px = gsp::pitch_for(nx);
    p->dp.Ps = gsp::sym_pitch_for(nx);
    const size_t cx = 2 * p->elem;
    const size_t sym_bytes = (size_t)(nz + 1) * (ny + 1) * (size_t)p->dp.Ps * p->elem;
    // Twiddles: the compiled forms W_{2N} (and, FP32, the column passes' (re, re, im, im)
    // copy); the runtime-length forms one table W_{2 n_q} per axis (double-float: 16 bytes
    // per entry, as FP64).
    const size_t tw_bytes = any ? (size_t)2 * (nx + ny + nz) * cx : (size_t)2 * N * cx;
    const size_t twc_bytes = dtype == POISSON_F32 && !any ? (size_t)2 * N * 4 * sizeof(float) : 0;
    const size_t w1_bytes = (size_t)max_batch * nz * ny * p->dp.Px * cx;
    const size_t w2_bytes = (size_t)max_batch * nz * 2 * ny * p->dp.Px * cx;
    p->ws_bytes = w1_bytes + 2 * w2_bytes;  // for max_batch densities
    p->table_bytes = sym_bytes + tw_bytes + twc_bytes;

    double *dA = nullptr, *dw = nullptr, *dtau = nullptr, *dgl = nullptr;
    auto fail = [&](cudaError_t err) {
        for (double *b : {dA, dw, dtau, dgl})
            if (b) cudaFree(b);
        free_plan(p);
        return map_cuda(err);
    };
    if ((e = cudaMalloc(&p->dp.sym, sym_bytes)) != cudaSuccess) return fail(e);
    if (p->ht.box && !any) {
        if ((e = cudaMalloc(&p->dp.symT, sym_bytes)) != cudaSuccess) return fail(e);
        p->table_bytes += sym_bytes;
    }
    if ((e = cudaMalloc(&p->dp.tw, tw_bytes)) != cudaSuccess) return fail(e);
    if (any) {
        p->dp.tw3[0] = p->dp.tw;
        p->dp.tw3[1] = static_cast<char *>(p->dp.tw) + (size_t)2 * nx * cx;
        p->dp.tw3[2] = static_cast<char *>(p->dp.tw3[1]) + (size_t)2 * ny * cx;
    }
    if ((e = cudaMalloc(&p->dp.w1, w1_bytes)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&p->dp.w2, w2_bytes)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&p->dp.w3, w2_bytes)) != cudaSuccess) return fail(e);
    if (twc_bytes) {
        if ((e = cudaMalloc(&p->dp.twc, twc_bytes)) != cudaSuccess) return fail(e);
    } else {
        p->dp.twc = p->dp.tw;
    }
    // Padding columns (kx > N) are carried along by the two-column passes but never used;
    // zeroed once so they hold finite values.
    if ((e = cudaMemset(p->dp.w1, 0, w1_bytes)) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(p->dp.w2, 0, w2_bytes)) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(p->dp.w3, 0, w2_bytes)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&p->dp.status, sizeof(int))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&p->dp.tail, 2 * sizeof(double) * max_batch)) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(p->dp.status, 0, sizeof(int))) != cudaSuccess) return fail(e);
    if (!any && gsp::xy_forms(N, dtype) != 1) {
        const size_t sync_bytes = sizeof(int) * (size_t)gsp::xy_sync_ints();
        if ((e = cudaMalloc(&p->dp.sync, sync_bytes)) != cudaSuccess) return fail(e);
        if ((e = cudaMemset(p->dp.sync, 0, sync_bytes)) != cudaSuccess) return fail(e);
    }
    if (p->ht.box && !any) {
        // The z warp forms read the symbol with kz innermost, which for the cube is the table
        // itself (it is symmetric); a box's map covers its transposed copy instead.
        void *natural = p->dp.sym;
        p->dp.sym = p->dp.symT;
        e = gsp::encode_tma_maps(p->dp);
        const CUtensorMap zw_sym = p->dp.tm_zw_sym;
        p->dp.sym = natural;
        if (e == cudaSuccess) e = gsp::encode_tma_maps(p->dp);
        p->dp.tm_zw_sym = zw_sym;
        if (e != cudaSuccess) return fail(e);
    } else if ((e = gsp::encode_tma_maps(p->dp)) != cudaSuccess) {
        return fail(e);
    }
    gsp::ForkPool *pool = nullptr;
    if ((e = gsp::fork_pool(p->device, &pool)) != cudaSuccess) return fail(e);

    // The arithmetic and kernel forms, timed on the zeroed workspace (the tables below are
    // built in the chosen arithmetic's format).
    if ((e = cudaMemset(p->dp.sym, 0, sym_bytes)) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(p->dp.tw, 0, tw_bytes)) != cudaSuccess) return fail(e);
    if ((e = gsp::autotune(p->dp, p->device)) != cudaSuccess) return fail(e);
    if ((e = upload_twiddles(p)) != cudaSuccess) return fail(e);

    // Symbol on the device, in FP64, from the per-axis factors (a box: one table per axis,
    // l_q A_j(tau_j l_q), Sec. 2; a runtime-length plan: n_q + 1 frequencies on axis q).
    const int nterms = (int)p->ht.tau.size();
    const bool box = p->ht.box;
    const bool three = box || any;  // one table per axis
    size_t nA3[3], off3[3], tot = 0;
    for (int q = 0; q < 3; ++q) {
        nA3[q] = (size_t)nterms * (n3[q] + 1);
        off3[q] = tot;
        tot += three ? nA3[q] : (q == 0 ? nA3[0] : 0);
    }
    if ((e = cudaMalloc(&dA, tot * sizeof(double))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&dtau, (size_t)nterms * sizeof(double))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&dgl, 32 * sizeof(double))) != cudaSuccess) return fail(e);
    {
        double gl[32];
        gsp::gauss_legendre16(gl, gl + 16);
        if ((e = cudaMemcpy(dgl, gl, sizeof gl, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
    }
    if (!three) {
        if ((e = cudaMemcpy(dtau, p->ht.tau.data(), (size_t)nterms * sizeof(double), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            return fail(e);
        if ((e = gsp::launch_axis_table(dtau, dgl, nterms, N, dA, 0)) != cudaSuccess) return fail(e);
        p->ht.A.resize(nA3[0]);  // the plan keeps the table for poisson_plan_axis_table
        if ((e = cudaMemcpy(p->ht.A.data(), dA, nA3[0] * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return fail(e);
    } else {
        std::vector<double> taul(nterms);
        p->ht.A3.resize(tot);
        for (int q = 0; q < 3; ++q) {
            for (int j = 0; j < nterms; ++j) taul[j] = p->ht.tau[j] * p->ht.l[q];
            if ((e = cudaMemcpy(dtau, taul.data(), (size_t)nterms * sizeof(double), cudaMemcpyHostToDevice)) !=
                cudaSuccess)
                return fail(e);
            if ((e = gsp::launch_axis_table(dtau, dgl, nterms, n3[q], dA + off3[q], 0)) != cudaSuccess) return fail(e);
            if ((e = cudaMemcpy(p->ht.A3.data() + off3[q], dA + off3[q], nA3[q] * sizeof(double),
                                cudaMemcpyDeviceToHost)) != cudaSuccess)
                return fail(e);
            for (size_t i = 0; i < nA3[q]; ++i) p->ht.A3[off3[q] + i] *= p->ht.l[q];
        }
        if ((e = cudaMemcpy(dA, p->ht.A3.data(), tot * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(e);
        p->ht.A.assign(p->ht.A3.begin(), p->ht.A3.begin() + nA3[0]);  // the x axis
    }
    if ((e = cudaMalloc(&dw, p->ht.w.size() * sizeof(double))) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(dw, p->ht.w.data(), p->ht.w.size() * sizeof(double),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e);
    const double scale = p->ht.lambda * p->ht.lambda / (8.0 * nx * ny * nz);
    e = three ? gsp::launch_symbol_table_box(p->dp, dA, dw, nterms, p->ht.C0, p->ht.C2, scale, p->ht.l, 0, 0)
              : gsp::launch_symbol_table(p->dp, dA, dw, nterms, p->ht.C0, p->ht.C2, scale, 0, 0);
    if (e != cudaSuccess) return fail(e);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e);
    cudaFree(dA);
    cudaFree(dw);
    cudaFree(dtau);
    cudaFree(dgl);
    dA = dw = dtau = dgl = nullptr;
    *out = p;
    return POISSON_OK;
}

extern "C" int poisson_plan_get_knob(poisson_plan p, int knob, int *value) {
    if (!p || !value) return POISSON_ERR_ARG;
    if (knob == POISSON_KNOB_Z_FORM) *value = p->dp.zform;
    else if (knob == POISSON_KNOB_Y_FORM) *value = p->dp.yform;
    else if (knob == POISSON_KNOB_X_FORM) *value = p->dp.xform;
    else if (knob == POISSON_KNOB_XY_FORM) *value = p->dp.xyform;
    else if (knob == POISSON_KNOB_CORRECTION) *value = p->correction;
    else if (knob == POISSON_KNOB_ARITH) *value = p->dp.arith;
    else return POISSON_ERR_ARG;
    return POISSON_OK;
}

// Recompute the plan's symbol octant from its kept per-axis factors with the correction
// placed as `literal` says (0 fused, 1 the unpadded transform pair), on the plan's device.
static int rebuild_symbol(poisson_plan p, int literal) {
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return map_cuda(e);
    if ((e = cudaSetDevice(p->device)) != cudaSuccess) return map_cuda(e);
    const int nterms = (int)p->ht.tau.size();
    const bool three = p->ht.box || p->dp.any;
    const std::vector<double> &A = three ? p->ht.A3 : p->ht.A;  // one table or one per axis
    double *dA = nullptr, *dw = nullptr;
    e = cudaMalloc(&dA, A.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dw, (size_t)nterms * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(dA, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(dw, p->ht.w.data(), (size_t)nterms * sizeof(double), cudaMemcpyHostToDevice);
    const double scale = p->ht.lambda * p->ht.lambda / (8.0 * p->dp.n3[0] * p->dp.n3[1] * p->dp.n3[2]);
    if (e == cudaSuccess)
        e = three ? gsp::launch_symbol_table_box(p->dp, dA, dw, nterms, p->ht.C0, p->ht.C2, scale, p->ht.l, literal, 0)
                  : gsp::launch_symbol_table(p->dp, dA, dw, nterms, p->ht.C0, p->ht.C2, scale, literal, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(dA);
    cudaFree(dw);
    cudaSetDevice(prev);
    return map_cuda(e);
}

extern "C" int poisson_plan_set_knob(poisson_plan p, int knob, int value) {
    if (!p) return POISSON_ERR_ARG;
    if (knob == POISSON_KNOB_CORRECTION) {
        if (value != 0 && value != 1) return POISSON_ERR_ARG;
        if (value == p->correction) return POISSON_OK;
        const int rc = rebuild_symbol(p, value);
        if (rc == POISSON_OK) p->correction = value;
        return rc;
    }
    if (knob == POISSON_KNOB_ARITH) {
        if (value != 0 && value != 1) return POISSON_ERR_ARG;
        if (value == 1 && p->dp.dtype != POISSON_F64) return POISSON_ERR_UNSUPPORTED;
        if (value == p->dp.arith) return POISSON_OK;
        // The twiddles and the symbol change format with the arithmetic; the workspace
        // needs nothing (every solve writes each buffer before reading it).
        const int prev = p->dp.arith, prev_z = p->dp.zform;
        p->dp.arith = value;
        if (p->dp.any || !(gsp::z_forms(p->dp.N, p->dp.dtype, value) >> p->dp.zform & 1)) p->dp.zform = 0;
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaSetDevice(p->device);
        if (e == cudaSuccess) e = upload_twiddles(p);
        cudaSetDevice(dev);
        int rc = map_cuda(e);
        if (rc == POISSON_OK) rc = rebuild_symbol(p, p->correction);
        if (rc != POISSON_OK) {
            p->dp.arith = prev;
            p->dp.zform = prev_z;
            cudaSetDevice(p->device);
            upload_twiddles(p);
            cudaSetDevice(dev);
            rebuild_symbol(p, p->correction);
        }
        return rc;
    }
    int forms, *field;
    const bool any = p->dp.any != 0;  // the runtime-length forms have one form per pass
    if (knob == POISSON_KNOB_Z_FORM) {
        forms = any ? 1 : gsp::z_forms(p->dp.N, p->dp.dtype, p->dp.arith);
        field = &p->dp.zform;
    } else if (knob == POISSON_KNOB_Y_FORM) {
        forms = any ? 1 : gsp::y_forms(p->dp.N, p->dp.dtype);
        field = &p->dp.yform;
    } else if (knob == POISSON_KNOB_X_FORM) {
        forms = any ? 1 : gsp::x_forms(p->dp.N, p->dp.dtype);
        field = &p->dp.xform;
    } else if (knob == POISSON_KNOB_XY_FORM) {
        forms = p->dp.sync ? gsp::xy_forms(p->dp.N, p->dp.dtype) : 1;
        field = &p->dp.xyform;
    } else {
        return POISSON_ERR_ARG;
    }
    if (value < 0 || value > (knob == POISSON_KNOB_Z_FORM ? 2 : 1)) return POISSON_ERR_ARG;
    if (!(forms >> value & 1)) return POISSON_ERR_UNSUPPORTED;
    *field = value;
    return POISSON_OK;
}

extern "C" int poisson_plan_destroy(poisson_plan p) {
    free_plan(p);
    return POISSON_OK;
}

static int check_solve_args(poisson_plan p, const void *rho, const void *u) {
    if (!p || !rho || !u) return POISSON_ERR_ARG;
    return POISSON_OK;
}

static void one(gsp::PtrArray &a, const void *ptr) {
    a.p[0] = ptr;
    for (int i = 1; i < gsp::kMaxBatch; ++i) a.p[i] = nullptr;
}

extern "C" int poisson_solve(poisson_plan p, const void *rho_d, void *u_d, void *stream) {
    int rc = check_solve_args(p, rho_d, u_d);
    if (rc) return rc;
    gsp::PtrArray in, out;
    one(in, rho_d);
    one(out, u_d);
    return map_cuda(gsp::launch_solve(p->dp, in, out, 1, (cudaStream_t)stream, nullptr));
}

// Slabs of the host-buffer solve's copy / x-pass pipeline.
constexpr int kSlabs = 8;

extern "C" int poisson_solve_host(poisson_plan p, const void *rho_h, void *u_h, void *stream) {
    int rc = check_solve_args(p, rho_h, u_h);
    if (rc) return rc;
    const int nx = p->dp.n3[0], ny = p->dp.n3[1], nz = p->dp.n3[2];
    const size_t n = (size_t)nx * ny * nz * p->elem;
    cudaError_t e;
    if (!p->stage_in) {
        if ((e = cudaMalloc(&p->stage_in, n)) != cudaSuccess) return map_cuda(e);
    }
    if (!p->stage_out) {
        if ((e = cudaMalloc(&p->stage_out, n)) != cudaSuccess) return map_cuda(e);
    }
    cudaStream_t s = (cudaStream_t)stream;
    gsp::PtrArray in, out;
    one(in, p->stage_in);
    one(out, p->stage_out);
    const bool fused = p->dp.xyform == 1 && p->dp.sync != nullptr;
    if (fused || nz % kSlabs != 0 || nz < 2 * kSlabs) {
        if ((e = cudaMemcpyAsync(p->stage_in, rho_h, n, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return map_cuda(e);
        if ((e = gsp::launch_solve(p->dp, in, out, 1, s, nullptr)) != cudaSuccess) return map_cuda(e);
        if ((e = cudaMemcpyAsync(u_h, p->stage_out, n, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return map_cuda(e);
        return map_cuda(cudaStreamSynchronize(s));
    }
    // Slab pipeline: the x and y passes transform each z-plane on its own (only the z pass
    // needs the whole volume), so the copy of slab k + 1 to the device runs while the x and
    // y forward passes transform slab k, and the copy of slab k back to the host while the
    // y and x inverse passes make slab k + 1.  Copies on the plan's copy stream, passes on
    // `stream`, one event per slab and direction.
    if (!p->copy_stream && (e = cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return map_cuda(e);
    if (!p->have_slab_events) {
        for (auto &ev : p->slab_ev)
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return map_cuda(e);
        p->have_slab_events = true;
    }
    cudaStream_t cs = p->copy_stream;
    cudaEvent_t *ev_in = p->slab_ev, *ev_out = p->slab_ev + kSlabs, start = p->slab_ev[2 * kSlabs];
    const int nzs = nz / kSlabs;  // planes per slab
    const size_t sb = (size_t)nzs * ny * nx * p->elem;
    // On an error part of the pipeline may already be queued: wait for both streams so
    // that no copy into or out of the staging buffers outlives the call.
    auto fail = [&](cudaError_t err) {
        cudaStreamSynchronize(cs);
        cudaStreamSynchronize(s);
        return map_cuda(err);
    };
    // The copies wait for the work already on `stream` (an earlier solve reading the
    // staging buffers).
    if ((e = cudaEventRecord(start, s)) != cudaSuccess || (e = cudaStreamWaitEvent(cs, start, 0)) != cudaSuccess)
        return map_cuda(e);
    for (int k = 0; k < kSlabs; ++k) {
        e = cudaMemcpyAsync(static_cast<char *>(p->stage_in) + k * sb, static_cast<const char *>(rho_h) + k * sb, sb,
                            cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ev_in[k], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_in[k], 0);
        if (e == cudaSuccess) e = gsp::launch_xy_slab(p->dp, p->stage_in, p->stage_out, k * nzs, nzs, s, true);
        if (e != cudaSuccess) return fail(e);
    }
    if ((e = gsp::launch_solve(p->dp, in, out, 1, s, nullptr, nullptr, 3)) != cudaSuccess) return fail(e);
    for (int k = 0; k < kSlabs; ++k) {
        e = gsp::launch_xy_slab(p->dp, p->stage_in, p->stage_out, k * nzs, nzs, s, false);
        if (e == cudaSuccess) e = cudaEventRecord(ev_out[k], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_out[k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(static_cast<char *>(u_h) + k * sb, static_cast<char *>(p->stage_out) + k * sb, sb,
                                cudaMemcpyDeviceToHost, cs);
        if (e != cudaSuccess) return fail(e);
    }
    // `stream` waits for the last copy, so that work issued after the call is ordered
    // after it, then the call returns once everything has finished.
    if ((e = cudaEventRecord(start, cs)) != cudaSuccess || (e = cudaStreamWaitEvent(s, start, 0)) != cudaSuccess)
        return fail(e);
    if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) return fail(e);
    return map_cuda(cudaStreamSynchronize(s));
}

// ---- slab decomposition of one solve ---------------------------------------------------------
// A rank of a P-way decomposition owns planes z0 .. z0 + nz - 1 of the density for the x and
// y passes and lines ky0 .. ky0 + nky - 1 of the y-spectrum for the z pass; between them the
// caller moves blocks of the plan's y-spectrum buffers (poisson_plan_spectrum).
static int slab_planes_ok(poisson_plan p, const void *ptr, int z0, int nz) {
    if (!p || !ptr) return POISSON_ERR_ARG;
    if (z0 < 0 || nz < 1 || z0 + nz > p->dp.n3[2]) return POISSON_ERR_ARG;
    return POISSON_OK;
}

extern "C" int poisson_slab_forward(poisson_plan p, const void *rho_slab_d, int z0, int nz, void *stream) {
    int rc = slab_planes_ok(p, rho_slab_d, z0, nz);
    if (rc) return rc;
    // The pass code offsets a whole-density pointer by the slab's first plane.
    const uintptr_t off = (uintptr_t)z0 * p->dp.n3[1] * p->dp.n3[0] * p->elem;
    const void *base = reinterpret_cast<const void *>(reinterpret_cast<uintptr_t>(rho_slab_d) - off);
    void *none = const_cast<void *>(base);
    return map_cuda(gsp::launch_xy_slab(p->dp, base, none, z0, nz, (cudaStream_t)stream, true));
}

extern "C" int poisson_slab_z(poisson_plan p, int ky0, int nky, void *stream) {
    if (!p || ky0 < 0 || nky < 1 || ky0 + nky > 2 * p->dp.n3[1]) return POISSON_ERR_ARG;
    return map_cuda(GSP_BY_ARITH(p->dp, gsp::z_lines, p->dp, ky0, nky, (cudaStream_t)stream));
}

extern "C" int poisson_slab_inverse(poisson_plan p, void *u_slab_d, int z0, int nz, void *stream) {
    int rc = slab_planes_ok(p, u_slab_d, z0, nz);
    if (rc) return rc;
    const uintptr_t off = (uintptr_t)z0 * p->dp.n3[1] * p->dp.n3[0] * p->elem;
    void *base = reinterpret_cast<void *>(reinterpret_cast<uintptr_t>(u_slab_d) - off);
    return map_cuda(gsp::launch_xy_slab(p->dp, base, base, z0, nz, (cudaStream_t)stream, false));
}

extern "C" int poisson_plan_spectrum(poisson_plan p, int which, void **ptr, size_t *plane_bytes, size_t *row_bytes) {
    if (!p || (which != 0 && which != 1) || !ptr) return POISSON_ERR_ARG;
    const size_t row = (size_t)p->dp.Px * 2 * p->elem;
    *ptr = which == 0 ? p->dp.w2 : p->dp.w3;
    if (row_bytes) *row_bytes = row;
    if (plane_bytes) *plane_bytes = row * 2 * p->dp.n3[1];
    return POISSON_OK;
}

extern "C" int poisson_solve_batched(int count, const poisson_plan *plans,
                                     const void *const *rho_d, void *const *u_d, void *stream) {
    if (count < 0) return POISSON_ERR_ARG;
    if (count == 0) return POISSON_OK;
    if (!plans || !rho_d || !u_d) return POISSON_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        int rc = check_solve_args(plans[i], rho_d[i], u_d[i]);
        if (rc) return rc;
        if (plans[i]->device != plans[0]->device) return POISSON_ERR_ARG;
    }
    // Group the entries by plan (first-appearance order); each group runs as grouped
    // launches of at most max_batch densities, groups on separate forked streams.
    std::vector<poisson_plan> order;
    std::vector<std::vector<int>> members;
    for (int i = 0; i < count; ++i) {
        size_t k = 0;
        while (k < order.size() && order[k] != plans[i]) ++k;
        if (k == order.size()) {
            order.push_back(plans[i]);
            members.emplace_back();
        }
        members[k].push_back(i);
    }
    cudaStream_t s = (cudaStream_t)stream;
    gsp::ForkPool *pool = nullptr;
    cudaError_t e = gsp::fork_pool(plans[0]->device, &pool);
    if (e != cudaSuccess) return map_cuda(e);
    const bool fork = order.size() > 1;
    if (fork && (e = cudaEventRecord(pool->fork, s)) != cudaSuccess) return map_cuda(e);
    for (size_t k = 0; k < order.size(); ++k) {
        const int slot = (int)(k % gsp::ForkPool::kStreams);
        cudaStream_t ts = fork ? pool->st[slot] : s;
        if (fork && (e = cudaStreamWaitEvent(ts, pool->fork, 0)) != cudaSuccess) return map_cuda(e);
        const gsp::DevicePlan &dp = order[k]->dp;
        const std::vector<int> &m = members[k];
        for (size_t c0 = 0; c0 < m.size(); c0 += (size_t)dp.max_batch) {
            const int n = (int)std::min(m.size() - c0, (size_t)dp.max_batch);
            gsp::PtrArray in, out;
            for (int i = 0; i < gsp::kMaxBatch; ++i) {
                in.p[i] = i < n ? rho_d[m[c0 + i]] : nullptr;
                out.p[i] = i < n ? u_d[m[c0 + i]] : nullptr;
            }
            if ((e = gsp::launch_solve(dp, in, out, n, ts, nullptr)) != cudaSuccess) return map_cuda(e);
        }
        if (fork) {
            if ((e = cudaEventRecord(pool->join[slot], ts)) != cudaSuccess) return map_cuda(e);
            if ((e = cudaStreamWaitEvent(s, pool->join[slot], 0)) != cudaSuccess) return map_cuda(e);
        }
    }
    return POISSON_OK;
}

extern "C" int poisson_solve_timed(poisson_plan p, const void *rho_d, void *u_d, void *stream,
                                   float *ms) {
    int rc = check_solve_args(p, rho_d, u_d);
    if (rc) return rc;
    if (!ms) return POISSON_ERR_ARG;
    cudaError_t e;
    if (!p->have_events) {
        for (int i = 0; i < 6; ++i)
            if ((e = cudaEventCreate(&p->ev[i])) != cudaSuccess) return map_cuda(e);
        p->have_events = true;
    }
    gsp::PtrArray in, out;
    one(in, rho_d);
    one(out, u_d);
    if ((e = gsp::launch_solve(p->dp, in, out, 1, (cudaStream_t)stream, p->ev)) != cudaSuccess)
        return map_cuda(e);
    if ((e = cudaEventSynchronize(p->ev[5])) != cudaSuccess) return map_cuda(e);
    for (int i = 0; i < 5; ++i)
        if ((e = cudaEventElapsedTime(&ms[i], p->ev[i], p->ev[i + 1])) != cudaSuccess)
            return map_cuda(e);
    return POISSON_OK;
}

extern "C" int poisson_solve_checked(poisson_plan p, const void *rho_d, void *u_d, double *eta,
                                     void *stream) {
    int rc = check_solve_args(p, rho_d, u_d);
    if (rc) return rc;
    if (!eta) return POISSON_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaMemsetAsync(p->dp.tail, 0, 2 * sizeof(double), s)) != cudaSuccess) return map_cuda(e);
    gsp::PtrArray in, out;
    one(in, rho_d);
    one(out, u_d);
    if ((e = gsp::launch_solve(p->dp, in, out, 1, s, nullptr, p->dp.tail)) != cudaSuccess) return map_cuda(e);
    double h[2] = {0.0, 0.0};
    if ((e = cudaMemcpyAsync(h, p->dp.tail, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return map_cuda(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return map_cuda(e);
    *eta = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : 0.0;
    return POISSON_OK;
}

extern "C" int poisson_solve_checked_batched(poisson_plan p, int count, const void *const *rho_d, void *const *u_d,
                                             double *eta, void *stream) {
    if (!p || !rho_d || !u_d || !eta || count < 1 || count > p->dp.max_batch) return POISSON_ERR_ARG;
    for (int i = 0; i < count; ++i)
        if (!rho_d[i] || !u_d[i]) return POISSON_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaMemsetAsync(p->dp.tail, 0, 2 * sizeof(double) * count, s)) != cudaSuccess) return map_cuda(e);
    gsp::PtrArray in, out;
    for (int i = 0; i < gsp::kMaxBatch; ++i) {
        in.p[i] = i < count ? rho_d[i] : nullptr;
        out.p[i] = i < count ? u_d[i] : nullptr;
    }
    if ((e = gsp::launch_solve(p->dp, in, out, count, s, nullptr, p->dp.tail)) != cudaSuccess) return map_cuda(e);
    double h[2 * gsp::kMaxBatch];
    if ((e = cudaMemcpyAsync(h, p->dp.tail, 2 * sizeof(double) * count, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return map_cuda(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return map_cuda(e);
    for (int i = 0; i < count; ++i) eta[i] = h[2 * i + 1] > 0.0 ? std::sqrt(h[2 * i] / h[2 * i + 1]) : 0.0;
    return POISSON_OK;
}

extern "C" int poisson_last_status(poisson_plan p, void *stream) {
    if (!p) return POISSON_ERR_ARG;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, p->dp.status, sizeof(int), cudaMemcpyDeviceToHost,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return map_cuda(e);
    if (h == 0) return POISSON_OK;
    e = cudaMemsetAsync(p->dp.status, 0, sizeof(int), (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return map_cuda(e);
    return (h & gsp::kStatusTimeoutBit) ? POISSON_ERR_TIMEOUT : POISSON_ERR_CUDA;
}

extern "C" int poisson_selftest_wait(poisson_plan p, long long polls, void *stream) {
    if (!p || polls < 1 || polls > (1ll << 24)) return POISSON_ERR_ARG;
    return map_cuda(gsp::launch_wait_selftest(p->dp, polls, (cudaStream_t)stream));
}

extern "C" int poisson_plan_info(poisson_plan p, double *delta, double *eps, int *n_terms,
                                 double *c0, double *c2, size_t *ws_bytes, size_t *table_bytes) {
    if (!p) return POISSON_ERR_ARG;
    if (delta) *delta = p->ht.delta;
    if (eps) *eps = p->ht.eps;
    if (n_terms) *n_terms = (int)p->ht.tau.size();
    if (c0) *c0 = p->ht.C0;
    if (c2) *c2 = p->ht.C2;
    if (ws_bytes) *ws_bytes = p->ws_bytes;
    if (table_bytes) *table_bytes = p->table_bytes;
    return POISSON_OK;
}

extern "C" int poisson_plan_gauss_sum(poisson_plan p, double *tau, double *w, int cap) {
    if (!p || cap < 0 || (cap > 0 && (!tau || !w))) return POISSON_ERR_ARG;
    const int n = std::min(cap, (int)p->ht.tau.size());
    for (int j = 0; j < n; ++j) {
        tau[j] = p->ht.tau[j];
        w[j] = p->ht.w[j];
    }
    return POISSON_OK;
}

extern "C" int poisson_plan_axis_table(poisson_plan p, double *a, size_t cap) {
    if (!p || (cap > 0 && !a)) return POISSON_ERR_ARG;
    const size_t n = std::min(cap, p->ht.A.size());
    if (n) std::memcpy(a, p->ht.A.data(), n * sizeof(double));
    return POISSON_OK;
}
