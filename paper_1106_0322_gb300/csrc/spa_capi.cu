// spa_capi.cu -- the host runtime behind include/spa.h.
//
// A context owns one region's genotype store and the device workspace of its sweeps.
// spa_run enqueues the whole sweep -- init, then per scale step: reweight, log-sum-exp /
// ESS, conditional resampling, proposal scales, M x (MH test of the previous move fused with
// the next proposal, likelihood), the last MH test with its commit, summaries -- on one stream, captures it once into a CUDA graph keyed by
// (T, N, M, config), and replays the graph for later sweeps of the same shape. The
// schedule and the seed live in device memory, so a replay only re-uploads them.
// Decisions that depend on data (resample or not) are taken on the device (a flag the
// resampling kernels read), so the host never waits inside a sweep.
#include <dlfcn.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/spa.h"
#include "spa_device.cuh"
#include "spa_internal.h"

using namespace spa;

namespace {

// Message of the last failed context-free call on this thread (fixed storage: setting it
// never allocates).
thread_local char g_thread_error[512] = {0};

void set_thread_error_str(const std::string& m) { std::snprintf(g_thread_error, sizeof(g_thread_error), "%s", m.c_str()); }

// Host-side fault injection for the failure-path tests: SPA_FAULT holds a comma-separated
// list of faults, read at every call that can inject one.
//   alloc       every device allocation of the library fails (SPA_ENOMEM)
//   nan_weight  a sweep's first log-weight is set to NaN after the initial weighting
//               (SPA_ENUMERIC from the device-side check of the log-sum-exp)
//   stall       every tensor-core likelihood launch first waits on a barrier that nothing
//               arrives at, so that bounded wait runs out after the context's wait limit
//               (SPA_ETIMEOUT); the kernel then drains its own copies and returns
// None of these faults, traps or hangs the GPU.
enum : int { FAULT_ALLOC = 1, FAULT_NAN_WEIGHT = 2, FAULT_STALL = 4 };

int fault_mask()
{
    const char* s = std::getenv("SPA_FAULT");
    if (!s || !*s) return 0;
    int m = 0;
    std::string v(s);
    size_t a = 0;
    while (a <= v.size()) {
        size_t b = v.find(',', a);
        if (b == std::string::npos) b = v.size();
        const std::string tok = v.substr(a, b - a);
        if (tok == "alloc") m |= FAULT_ALLOC;
        if (tok == "nan_weight") m |= FAULT_NAN_WEIGHT;
        if (tok == "stall") m |= FAULT_STALL;
        a = b + 1;
    }
    return m;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count)
{
    *p = nullptr;
    if (fault_mask() & FAULT_ALLOC) return cudaErrorMemoryAllocation;
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

template <typename T>
void dfree(T*& p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

// Round x up to a multiple of m.
inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

struct Workspace {
    int64_t N = 0, N_pad = 0;
    float *beta = nullptr, *beta_p = nullptr, *scale = nullptr;
    __nv_bfloat16* A = nullptr;
    CUtensorMap mapA, mapAt;  // the particle operand (64-column boxes; narrow last k-block)
    int BN = 0;               // n-tile width of the likelihood kernel's tile configuration
    int cfg = -1;             // the likelihood kernel's tile configuration (tuned per shape)
    int cfg_source = 0;       // where it came from: 0 fixed (environment, context, small n), 1 table, 2 timed
    float2* lpt_p = nullptr;  // compensated log-prior term sums of the proposals
    float2* ydq = nullptr;    // the proposals' linear log-likelihood term beta' . v
    float2 *llq = nullptr, *lpq = nullptr, *llq_tmp = nullptr, *lpq_tmp = nullptr;  // MH state pairs
    double *ll = nullptr, *logw = nullptr, *W = nullptr;  // ll: FP64 log-likelihood output of the entry points
    float* Wf = nullptr;
    uint32_t* wfix = nullptr;
    double *cum = nullptr, *lambda = nullptr, *lse_scratch = nullptr;
    uint32_t* keysT = nullptr;  // [p][N] order-preserving keys of beta for the summaries
    float* lu = nullptr;        // [2][N_pad] log U of the pending proposals' MH tests
    float* WfS = nullptr;       // the weights the summaries of a step read, copied beside the keys
    uint32_t* wfixS = nullptr;
    unsigned int* lse_counter = nullptr;
    float4* colpart = nullptr;
    float* h = nullptr;  // MALA step h = lambda p^(-1/6)
    float* partial = nullptr;
    int32_t* idx = nullptr;
    int* flag = nullptr;
    float* eta = nullptr;  // gradient path scratch, allocated on first use
    float* grad = nullptr;
    // MALA: log-likelihood gradient of the current and the proposed particles, forward residual sums
    float* gl = nullptr;
    float* gl_p = nullptr;
    float2* fwd = nullptr;
    // tensor-core adjoint: residuals r (BF16 hi | lo), their row sums, C = R G partials
    __nv_bfloat16* R = nullptr;
    float* rsum = nullptr;
    float* gpart = nullptr;
    CUtensorMap mapR;
};

struct RunBufs {
    int64_t T = 0;
    int nq = 0, nd = 0;
    double *sched = nullptr, *mean = nullptr, *quant = nullptr, *conc = nullptr, *ess = nullptr, *logz = nullptr,
           *accrate = nullptr;
    unsigned long long* acc = nullptr;
    uint8_t* res = nullptr;
    uint64_t* seed = nullptr;
    float* best = nullptr;  // [T][p] each step's particle of highest posterior density (map_path)
    float4* stepk = nullptr;  // [T] the move kernels' constants of each scale (launch_step_constants)
    ReweightK* rk = nullptr;  // [T] the reweighting kernel's constants of each step
};

struct GraphKey {
    int64_t T = -1, N = -1;
    int32_t M = -1;
    int fault = 0;  // injected faults captured into the graph
    spa_config cfg;
    bool operator==(const GraphKey& o) const
    {
        return T == o.T && N == o.N && M == o.M && fault == o.fault &&
               std::memcmp(&cfg, &o.cfg, sizeof(spa_config)) == 0;
    }
};

}  // namespace

namespace spa {
void set_thread_error(const char* msg, int64_t value)
{
    if (value >= 0)
        std::snprintf(g_thread_error, sizeof(g_thread_error), "%s%lld", msg, (long long)value);
    else
        std::snprintf(g_thread_error, sizeof(g_thread_error), "%s", msg);
}
}  // namespace spa

struct spa_ctx {
    int64_t n = 0, p = 0;
    int Kp = 0;
    double nu = 1.0;
    PriorArgs pr{1.0f, 0};
    int device = 0, num_sms = 0;
    // SMs the tensor-core launches are sized for (0: all of them). A batch sets it while it
    // captures its regions' sweeps side by side (see batch_plan_sms); buffers are always
    // sized for all SMs, which is the largest any plan needs.
    int plan_sms = 0;
    cudaStream_t own_stream = nullptr;
    // the key transpose and the summaries of step t run on side_stream beside step t + 1
    // (fork after the step's moves; the next step waits for the transpose before it
    // rewrites the weights, and the sweep's end joins the last summaries)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_keys = nullptr, ev_join = nullptr;
    spa_config cfg;
    std::string err;
    // genotype store
    int8_t* G = nullptr;
    uint8_t* y = nullptr;
    unsigned long long* sums = nullptr;
    double *mean = nullptr, *sd = nullptr, *v = nullptr, *unit_c = nullptr;
    float4* unit_k = nullptr;  // the move kernels' constants at c = 1 (packing at fixed scale)
    float *l2e_s = nullptr, *mean_f = nullptr, *Xf = nullptr;
    float* colf = nullptr;  // [3p]: 1/s_j, v_j, v_j log2(e) (FP32)
    __nv_bfloat16* Gbf = nullptr;
    CUtensorMap mapB, mapBt;  // the genotype operand for n-tiles of mapB_BN (64 columns; narrow last k-block)
    int mapB_BN = 0;
    __nv_bfloat16* GT = nullptr;  // [p][n_r] for the adjoint
    float* yv = nullptr;
    float* XT2 = nullptr;  // [p][n] X^T log2(e) for the single-coordinate kernel
    uint32_t* ybits = nullptr;  // y as a bitmask, one word per 32 individuals
    int64_t ywords = 0;
    int64_t n_r = 0;
    CUtensorMap mapGT;
    int mapGT_BN = 0;
    uint32_t* d_err = nullptr;
    Workspace ws;
    RunBufs rb;
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey;
    uint64_t gen = 0;  // bumped whenever captured work may refer to stale buffers or config
    int64_t graph_launches = 0;
    int64_t last_launches = 0;
    int64_t best_T = 0;        // steps recorded in rb.best by the last run (0: none)
    int map_rounds = 0;        // Jacobi rounds after round 0 of the last spa_map_path
    float* lip = nullptr;      // ||X||_2^2 / 4 for the MAP solver
    bool lip_ok = false;
    uint64_t wait_ns = 0;      // limit of the tensor-core kernels' bounded waits (0: the default)
    int tile_cfg = -1;         // likelihood tile configuration fixed by spa_set_tile_config (-1: tuned)
    int fault = 0;             // faults injected into the current sweep graph (SPA_FAULT)

    cudaStream_t stream() const { return cfg.stream ? static_cast<cudaStream_t>(cfg.stream) : own_stream; }
};

namespace {

int fail(spa_ctx* c, int code, const std::string& msg)
{
    if (c)
        c->err = msg;
    else
        set_thread_error_str(msg);
    return code;
}

int cuda_fail(spa_ctx* c, cudaError_t e, const char* what)
{
    return fail(c, e == cudaErrorMemoryAllocation ? SPA_ENOMEM : SPA_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

int check_device(spa_ctx* c)
{
    int dev = 0;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, dev), "cudaGetDeviceProperties");
    if (prop.major != 10)
        return fail(c, SPA_EUNSUPPORTED, "the library is built for sm_103a (compute capability 10.x)");
    CK(tc_init_attributes(), "tensor-core kernel attributes");
    CK(smc_init_attributes(), "summaries kernel attributes");
    CK(map_init_attributes(), "MAP kernel attributes");
    if (c) {
        c->device = dev;
        c->num_sms = prop.multiProcessorCount;
    }
    return SPA_OK;
}

int map_device_error(spa_ctx* c, uint32_t e)
{
    if (e == 0) return SPA_OK;
    if (e & DERR_TIMEOUT) return fail(c, SPA_ETIMEOUT, "a bounded device wait gave up");
    if (e & DERR_INPUT) return fail(c, SPA_EINVAL, "invalid input data (genotype not in {0,1,2}, phenotype not in {0,1}, or a monomorphic marker)");
    if (e & DERR_NONFINITE) return fail(c, SPA_ENUMERIC, "non-finite log-likelihood or log-weight");
    if (e & DERR_ESS) return fail(c, SPA_ENUMERIC, "effective sample size below 1");
    return fail(c, SPA_ECUDA, "unknown device error");
}

int read_error_word(spa_ctx* c)
{
    uint32_t e = 0;
    CK(cudaMemcpyAsync(&e, c->d_err, sizeof(e), cudaMemcpyDeviceToHost, c->stream()), "read error word");
    CK(cudaStreamSynchronize(c->stream()), "stream synchronize");
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), c->stream()), "reset error word");
    return map_device_error(c, e);
}

void free_workspace(Workspace& w)
{
    dfree(w.beta); dfree(w.beta_p); dfree(w.scale); dfree(w.A);
    dfree(w.lpt_p); dfree(w.ydq); dfree(w.llq); dfree(w.lpq); dfree(w.llq_tmp); dfree(w.lpq_tmp);
    dfree(w.ll); dfree(w.logw); dfree(w.W); dfree(w.Wf); dfree(w.wfix); dfree(w.cum); dfree(w.keysT); dfree(w.WfS); dfree(w.wfixS); dfree(w.lu); dfree(w.colpart); dfree(w.lambda); dfree(w.h);
    dfree(w.lse_scratch); dfree(w.lse_counter);
    dfree(w.partial); dfree(w.idx); dfree(w.flag); dfree(w.eta); dfree(w.grad);
    dfree(w.gl); dfree(w.gl_p); dfree(w.fwd); dfree(w.R); dfree(w.rsum); dfree(w.gpart);
    w.N = w.N_pad = 0;
    w.BN = 0;
    w.cfg = -1;
}

void free_runbufs(RunBufs& r)
{
    dfree(r.sched); dfree(r.mean); dfree(r.quant); dfree(r.conc); dfree(r.ess); dfree(r.logz); dfree(r.accrate);
    dfree(r.acc); dfree(r.res); dfree(r.seed); dfree(r.best); dfree(r.stepk); dfree(r.rk);
    r.T = 0;
}

// Drop the context's own sweep graph. bump: the buffers or the config it used are about
// to change, so graphs of batches holding this context become stale too.
void drop_graph(spa_ctx* c, bool bump = true)
{
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    if (bump) ++c->gen;
    c->gkey = GraphKey();
}

int ensure_mapB(spa_ctx* c, int BN)
{
    if (c->mapB_BN == BN) return SPA_OK;
    const int tw = tc_plan(c->n, (int)c->p, 128, c->num_sms, BN == 128 ? 1 : 0).tw;  // tw depends on p only
    if (!tc_make_map_B(&c->mapB, c->Gbf, c->n, c->Kp, BN) ||
        !tc_make_map_B_tail(&c->mapBt, c->Gbf, c->n, c->Kp, BN, tw))
        return fail(c, SPA_ECUDA, "cuTensorMapEncodeTiled failed for the genotype operand");
    c->mapB_BN = BN;
    return SPA_OK;
}

// ----------------------------------------------------------- likelihood tile tuner
// The tile configuration of the likelihood kernel (n-tile width, G stages, epilogue warps)
// sets how evenly the (particle-tile, n-tile) units spread over the SMs, how often each
// particle tile is streamed again and how the epilogue hides its latencies. The result does
// not depend on it: the partial sums are per 32-individual chunk whatever the tile. A shape
// (device, N_pad, n, p) takes, in this order: SPA_TILE_CONFIG=0..6 (or SPA_LOGLIK_BN=256|128,
// configurations 0|1) from the environment; a configuration fixed on the context
// (spa_set_tile_config); the nearest entry of the tile table, a JSON file written by the
// library's tuning script on a GB300 (SPA_TILE_TABLE, else tuning/loglik_tiles.json beside the
// package); else every valid configuration is timed once per process on the context's
// stream (3 warm-up and 10 timed launches each, CUDA events) and the fastest is kept.
struct TileEntry {
    int64_t n, p, N_pad;
    int cfg;
};

std::string library_dir()
{
    Dl_info info;
    if (dladdr(reinterpret_cast<void*>(&spa_config_default), &info) == 0 || !info.dli_fname) return ".";
    std::string f(info.dli_fname);
    const size_t k = f.find_last_of('/');
    return k == std::string::npos ? "." : f.substr(0, k);
}

// The integer after "key": inside [b, e) of s, or -1.
int64_t json_int(const std::string& s, size_t b, size_t e, const char* key)
{
    const std::string k = std::string("\"") + key + "\"";
    size_t i = s.find(k, b);
    if (i == std::string::npos || i >= e) return -1;
    i = s.find(':', i + k.size());
    if (i == std::string::npos || i >= e) return -1;
    return std::strtoll(s.c_str() + i + 1, nullptr, 10);
}

// The table's entries: the objects of its "entries" list with integer n, p, N_pad and config.
const std::vector<TileEntry>& tile_table()
{
    static std::vector<TileEntry> table;
    static std::once_flag once;
    std::call_once(once, [] {
        const char* env = std::getenv("SPA_TILE_TABLE");
        const std::string path = env ? std::string(env) : library_dir() + "/../tuning/loglik_tiles.json";
        FILE* f = std::fopen(path.c_str(), "rb");
        if (!f) return;
        std::string s;
        char buf[4096];
        size_t got;
        while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) s.append(buf, got);
        std::fclose(f);
        size_t i = s.find("\"entries\"");
        while (i != std::string::npos) {
            const size_t b = s.find('{', i);
            if (b == std::string::npos) break;
            const size_t e = s.find('}', b);
            if (e == std::string::npos) break;
            TileEntry t{json_int(s, b, e, "n"), json_int(s, b, e, "p"), json_int(s, b, e, "N_pad"),
                        (int)json_int(s, b, e, "config")};
            if (t.n > 0 && t.p > 0 && t.N_pad > 0 && t.cfg >= 0 && t.cfg < TC_CONFIGS) table.push_back(t);
            i = e + 1;
        }
    });
    return table;
}

// The table's configuration for the nearest shape (sum of the absolute log ratios of n, p + 1
// and N_pad at most 0.75), if it is valid for this shape's kernel mode; else -1.
int table_config(int64_t n, int64_t p, int64_t N_pad, bool resident)
{
    const std::vector<TileEntry>& t = tile_table();
    double best = 1e30;
    int cfg = -1;
    for (const TileEntry& e : t) {
        if ((e.p + 1 <= 256) != resident) continue;  // the same kernel mode
        const double d = std::fabs(std::log((double)n / (double)e.n)) +
                         std::fabs(std::log((double)(p + 1) / (double)(e.p + 1))) +
                         std::fabs(std::log((double)N_pad / (double)e.N_pad));
        if (d < best) {
            best = d;
            cfg = e.cfg;
        }
    }
    return (best <= 0.75 && tc_config_valid(cfg, p)) ? cfg : -1;
}

int tune_tile(spa_ctx* c)
{
    Workspace& w = c->ws;
    const bool resident = tc_plan_resident(tc_plan(c->n, (int)c->p, w.N_pad, c->num_sms, 0));
    if (const char* env = std::getenv("SPA_TILE_CONFIG")) {
        const int v = std::atoi(env);
        if (tc_config_valid(v, c->p)) {
            w.cfg_source = 0;
            return v;
        }
    }
    if (const char* env = std::getenv("SPA_LOGLIK_BN")) {
        const int v = std::atoi(env);
        if (v == 128 || v == 256) {
            w.cfg_source = 0;
            return v == 128 ? 1 : 0;
        }
    }
    if (tc_config_valid(c->tile_cfg, c->p)) {
        w.cfg_source = 0;
        return c->tile_cfg;
    }
    if (c->n <= 128) {
        w.cfg_source = 0;
        return 1;
    }
    const int tab = table_config(c->n, c->p, w.N_pad, resident);
    if (tab >= 0) {
        w.cfg_source = 1;
        return tab;
    }
    w.cfg_source = 2;
    static std::mutex mu;
    static std::map<std::tuple<int, int64_t, int64_t, int64_t>, int> cache;
    const auto key = std::make_tuple(c->device, w.N_pad, c->n, c->p);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    cudaStream_t st = c->stream();
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return 0;
    }
    int best = 0;
    float best_ms = -1.0f;
    for (int cfg = 0; cfg < TC_CONFIGS; ++cfg) {
        if (!tc_config_valid(cfg, c->p)) continue;
        const TcPlan plan = tc_plan(c->n, (int)c->p, w.N_pad, c->num_sms, cfg);
        TcMaps m;
        m.A = w.mapA;
        m.At = w.mapAt;
        m.Araw = w.A;
        if (!tc_make_map_B(&m.B, c->Gbf, c->n, c->Kp, plan.BN) ||
            !tc_make_map_B_tail(&m.Bt, c->Gbf, c->n, c->Kp, plan.BN, plan.tw))
            continue;
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < 3 && e == cudaSuccess; ++k)
            e = launch_loglik_tc(m, plan, c->n, c->Kp, c->ybits, w.partial, w.N_pad, c->d_err, st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int k = 0; k < 10 && e == cudaSuccess; ++k)
            e = launch_loglik_tc(m, plan, c->n, c->Kp, c->ybits, w.partial, w.N_pad, c->d_err, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) continue;
        if (best_ms < 0.0f || ms < best_ms) {
            best_ms = ms;
            best = cfg;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = best;
    return best;
}

int ensure_workspace(spa_ctx* c, int64_t N)
{
    Workspace& w = c->ws;
    if (w.N == N) return SPA_OK;
    drop_graph(c);
    free_workspace(w);
    const int64_t p = c->p;
    const int64_t N_pad = round_up(N, 128);
    const TcPlan plan = tc_plan(c->n, (int)p, N_pad, c->num_sms);  // n_parts does not depend on BN
    const int64_t simt_parts = (c->n + SIMT_TILE_N - 1) / SIMT_TILE_N;
    const int64_t parts = plan.n_parts > simt_parts ? plan.n_parts : simt_parts;
    const int64_t nblk = (N + 255) / 256;
    cudaError_t e = cudaSuccess;
#define WA(ptr, cnt) \
    if (e == cudaSuccess) e = dalloc(&w.ptr, (size_t)(cnt))
    WA(beta, N * p);
    WA(beta_p, N * p);
    WA(scale, 3 * p);  // RW: sigma; MALA: D, sqrt(D), 1/D
    WA(A, N_pad * 2 * c->Kp);
    WA(lpt_p, N); WA(ydq, N); WA(llq, N); WA(lpq, N); WA(llq_tmp, N); WA(lpq_tmp, N);
    WA(ll, N); WA(logw, N); WA(W, N); WA(Wf, N); WA(wfix, N);
    WA(keysT, N * p);
    WA(WfS, N); WA(wfixS, N);
    WA(lu, 2 * N_pad);
    WA(cum, N + nblk + 1);
    WA(colpart, (int64_t)COLSTAT_SPLITS * p);
    WA(lambda, 1);
    WA(h, 1);
    WA(lse_scratch, LSE_SCRATCH);
    WA(lse_counter, 1);
    WA(partial, parts * N_pad);
    WA(idx, N);
    WA(flag, 1);
#undef WA
    if (e != cudaSuccess) {
        free_workspace(w);
        return cuda_fail(c, e, "workspace allocation");
    }
    // The GEMM operand's padding (columns p+1..Kp-1 of both halves, rows N..N_pad-1) stays zero.
    CK(cudaMemsetAsync(w.A, 0, sizeof(__nv_bfloat16) * (size_t)(N_pad * 2 * c->Kp), c->stream()), "memset A");
    CK(cudaMemsetAsync(w.partial, 0, sizeof(float) * (size_t)(parts * N_pad), c->stream()), "memset partial");
    CK(cudaMemsetAsync(w.flag, 0, sizeof(int), c->stream()), "memset flag");
    CK(cudaMemsetAsync(w.lse_counter, 0, sizeof(unsigned int), c->stream()), "memset counter");
    if (!tc_make_map_A(&w.mapA, w.A, N_pad, c->Kp) || !tc_make_map_A_tail(&w.mapAt, w.A, N_pad, c->Kp, plan.tw)) {
        free_workspace(w);
        return fail(c, SPA_ECUDA, "cuTensorMapEncodeTiled failed for the particle operand");
    }
    w.N = N;
    w.N_pad = N_pad;
    w.cfg = tune_tile(c);
    w.BN = tc_config_bn(w.cfg);
    return ensure_mapB(c, w.BN);
}

int ensure_adjoint_buffers(spa_ctx* c)
{
    Workspace& w = c->ws;
    if (w.R) return SPA_OK;
    const AdjPlan a = adj_plan((int)c->p, c->n, w.N_pad, c->num_sms);
    const TcPlan plan = tc_plan(c->n, (int)c->p, w.N_pad, c->num_sms);
    cudaError_t e = dalloc(&w.R, (size_t)(w.N_pad * 2 * a.n_r));
    if (e == cudaSuccess) e = dalloc(&w.rsum, (size_t)(plan.n_parts * w.N_pad));
    if (e == cudaSuccess) e = dalloc(&w.gpart, (size_t)(a.ksplit * w.N_pad * c->p));
    if (e == cudaSuccess && !w.gl_p) e = dalloc(&w.gl_p, (size_t)(w.N * c->p));
    if (e != cudaSuccess) return cuda_fail(c, e, "adjoint buffers");
    // residual columns n..n_r-1 and rows N..N_pad-1 stay zero
    CK(cudaMemsetAsync(w.R, 0, sizeof(__nv_bfloat16) * (size_t)(w.N_pad * 2 * a.n_r), c->stream()), "memset R");
    if (!adj_make_map_R(&w.mapR, w.R, w.N_pad, a.n_r)) return fail(c, SPA_ECUDA, "cuTensorMapEncodeTiled failed for R");
    if (c->mapGT_BN != a.BN2) {
        if (!adj_make_map_GT(&c->mapGT, c->GT, (int)c->p, a.n_r, a.BN2))
            return fail(c, SPA_ECUDA, "cuTensorMapEncodeTiled failed for G^T");
        c->mapGT_BN = a.BN2;
    }
    return SPA_OK;
}

int ensure_mala_buffers(spa_ctx* c)
{
    Workspace& w = c->ws;
    if (c->cfg.precision == SPA_PREC_SPLIT_BF16) {
        int rc = ensure_adjoint_buffers(c);
        if (rc != SPA_OK) return rc;
    }
    const bool plain = c->cfg.precision != SPA_PREC_SPLIT_BF16;
    if (w.gl && (w.eta || !plain)) return SPA_OK;
    const int64_t N = w.N, p = c->p, n = c->n;
    const int64_t tiles = (n + SIMT_TILE_N - 1) / SIMT_TILE_N;
    cudaError_t e = cudaSuccess;
    if (!w.gl) e = dalloc(&w.gl, (size_t)(N * p));
    if (e == cudaSuccess && !w.gl_p) e = dalloc(&w.gl_p, (size_t)(N * p));
    if (e == cudaSuccess && !w.fwd) e = dalloc(&w.fwd, (size_t)N);
    if (e == cudaSuccess && plain && !w.eta) e = dalloc(&w.eta, (size_t)(N * n + tiles * N));
    if (e == cudaSuccess && plain && !w.grad) e = dalloc(&w.grad, (size_t)(N * p));
    if (e != cudaSuccess) return cuda_fail(c, e, "MALA buffers");
    return SPA_OK;
}

int ensure_runbufs(spa_ctx* c, int64_t T)
{
    RunBufs& r = c->rb;
    const int nq = c->cfg.n_quantiles, nd = c->cfg.n_deltas;
    if (r.T == T && r.nq == nq && r.nd == nd) return SPA_OK;
    drop_graph(c);
    free_runbufs(r);
    const int64_t p = c->p;
    cudaError_t e = cudaSuccess;
#define RA(ptr, cnt) \
    if (e == cudaSuccess) e = dalloc(&r.ptr, (size_t)(cnt))
    RA(sched, T);
    RA(mean, T * p);
    RA(quant, T * p * (nq > 0 ? nq : 1));
    RA(conc, T * p * (nd > 0 ? nd : 1));
    RA(ess, T); RA(logz, T); RA(accrate, T);
    RA(acc, T + 1);
    RA(res, T);
    RA(seed, 1);
    RA(best, T * p);
    RA(stepk, T);
    RA(rk, T);
#undef RA
    if (e != cudaSuccess) {
        free_runbufs(r);
        return cuda_fail(c, e, "run buffer allocation");
    }
    r.T = T;
    r.nq = nq;
    r.nd = nd;
    return SPA_OK;
}

// --------------------------------------------------------------------- the sweep
struct Enq {
    spa_ctx* c;
    cudaStream_t st;
    int64_t launches = 0;
    cudaError_t e = cudaSuccess;
    void ck(cudaError_t x)
    {
        if (e == cudaSuccess) e = x;
        ++launches;
    }
};

// gradient of the log-likelihood at the packed particles (beta_p / A) into out, on the
// tensor cores: residual likelihood pass, C = R G, finish. Also leaves the softplus
// partials of those particles in w.partial.
int plan_sm_count(const spa_ctx* c) { return c->plan_sms > 0 ? c->plan_sms : c->num_sms; }

TcPlan plan_of(const spa_ctx* c) { return tc_plan(c->n, (int)c->p, c->ws.N_pad, plan_sm_count(c), c->ws.cfg); }

TcMaps maps_of(const spa_ctx* c)
{
    TcMaps m;
    m.A = c->ws.mapA;
    m.At = c->ws.mapAt;
    m.Araw = c->ws.A;
    m.B = c->mapB;
    m.Bt = c->mapBt;
    return m;
}

// The adjoint's second half after a residual likelihood pass: C = R G, then the gradient.
void enq_grad_tail(Enq& q, float* out, const float* Bsrc, double cs, int64_t N)
{
    spa_ctx* c = q.c;
    Workspace& w = c->ws;
    const TcPlan plan = plan_of(c);
    // the K-split from all SMs whatever plan_sm_count says: it sets how the FP32 partial sums
    // over individuals are grouped, so a batch's gradients stay those of a single run
    const AdjPlan a = adj_plan((int)c->p, c->n, w.N_pad, c->num_sms);
    q.ck(launch_adjoint_tc(w.mapR, c->mapGT, a, (int)c->p, w.gpart, w.N_pad, c->d_err, q.st, c->wait_ns,
                           c->plan_sms > 0 ? c->plan_sms : 0, /*r_last_use_hint=*/c->plan_sms == 0));
    q.ck(launch_grad_finish(w.gpart, a.ksplit, w.rsum, plan.n_parts, w.N_pad, N, (int)c->p, c->mean_f, c->colf, Bsrc,
                            c->pr, cs, out, q.st));
}

void enq_grad_tc(Enq& q, float* out, const float* Bsrc, double cs, int64_t N)
{
    spa_ctx* c = q.c;
    Workspace& w = c->ws;
    const AdjPlan a = adj_plan((int)c->p, c->n, w.N_pad, c->num_sms);
    ResidArgs ra{w.R, a.n_r, w.rsum};
    q.ck(launch_loglik_tc(maps_of(c), plan_of(c), c->n, c->Kp, c->ybits, w.partial, w.N_pad, c->d_err, q.st, &ra,
                          c->wait_ns, c->fault & FAULT_STALL));
    enq_grad_tail(q, out, Bsrc, cs, N);
}

// log-likelihood of the current proposals (beta_p) into the partial sums
void enq_loglik(Enq& q)
{
    spa_ctx* c = q.c;
    Workspace& w = c->ws;
    if (c->cfg.precision == SPA_PREC_SPLIT_BF16) {
        q.ck(launch_loglik_tc(maps_of(c), plan_of(c), c->n, c->Kp, c->ybits, w.partial, w.N_pad, c->d_err, q.st,
                              nullptr, c->wait_ns, c->fault & FAULT_STALL));
    } else {
        q.ck(launch_loglik_simt(w.beta_p, c->Xf, c->y, w.N, c->n, (int)c->p, w.partial, w.N_pad, q.st));
    }
}

// MH state of the context's particles; partial units are ln 2 * nats on the tensor-core
// path and nats on the FP32 path.
MhState mh_state(spa_ctx* c, unsigned long long* acc)
{
    Workspace& w = c->ws;
    const bool tc = c->cfg.precision == SPA_PREC_SPLIT_BF16;
    MhState m;
    m.llq = w.llq;
    m.lpq = w.lpq;
    m.lpt_p = w.lpt_p;
    m.ydq = w.ydq;
    m.partial = w.partial;
    m.n_parts = tc ? plan_of(c).n_parts : (int)((c->n + SIMT_TILE_N - 1) / SIMT_TILE_N);
    m.ld_part = w.N_pad;
    m.sp_scale_d = tc ? LN2 : 1.0;
    m.sp_scale = (float)m.sp_scale_d;
    m.acc_count = acc;
    m.lu = w.lu;
    m.ld_lu = w.N_pad;
    return m;
}

MoveArgs move_args(spa_ctx* c, unsigned long long* acc)
{
    Workspace& w = c->ws;
    const bool tc = c->cfg.precision == SPA_PREC_SPLIT_BF16;
    MoveArgs a;
    a.beta = w.beta;
    a.beta_p = w.beta_p;
    a.A = tc ? w.A : nullptr;
    a.ldA = 2 * c->Kp;
    a.Kp = c->Kp;
    a.lpt_p = w.lpt_p;
    a.ydq = w.ydq;
    a.sigma = w.scale;
    a.sqrt_D = w.scale + c->p;
    a.inv_D = w.scale + 2 * c->p;
    a.l2e_over_s = c->l2e_s;
    a.mean_f = c->mean_f;
    a.vy = c->colf + (tc ? 2 : 1) * c->p;
    a.mh = mh_state(c, acc);
    a.gl = w.gl;
    a.gl_p = w.gl_p;
    a.fwd = w.fwd;
    a.h = w.h;
    return a;
}

void enq_resample(Enq& q, int t)
{
    spa_ctx* c = q.c;
    Workspace& w = c->ws;
    q.ck(launch_resample_index(w.W, w.N, w.cum, w.idx, w.flag, t, c->rb.seed, 0.0, q.st));
    q.launches += 2;  // local sums, carries and search
    const bool mala = c->cfg.move_kind == SPA_MOVE_MALA;
    q.ck(launch_gather(w.idx, w.beta, w.beta_p, w.llq, w.lpq, w.llq_tmp, w.lpq_tmp, mala ? w.gl : nullptr,
                       mala ? w.gl_p : nullptr, w.N, (int)c->p, w.flag, q.st));
    WeightArrays wa{w.logw, w.W, w.Wf, w.wfix};
    q.ck(launch_copyback(w.beta, w.beta_p, w.llq, w.lpq, w.llq_tmp, w.lpq_tmp, mala ? w.gl : nullptr,
                         mala ? w.gl_p : nullptr, wa, w.N, (int)c->p, w.flag, q.st));
}

void enq_colstats(Enq& q, int t)
{
    spa_ctx* c = q.c;
    Workspace& w = c->ws;
    const int kind = c->cfg.move_kind == SPA_MOVE_MALA ? 1 : 0;
    q.ck(launch_colstats(w.beta, w.Wf, w.N, (int)c->p, w.colpart, w.scale, kind, c->cfg.rw_scale,
                         kind ? w.lambda : nullptr, c->cfg.sd_floor, c->rb.sched, t, kind ? w.h : nullptr, q.st));
    ++q.launches;  // two kernels
}

// A likelihood evaluation inside a sweep: of the initial prior draws (t = 0) or of a move's
// proposals. Both are of the packed particles (beta_p and the GEMM rows A); on the MALA path
// they also give the log-likelihood gradient, into gl (the draws) or gl_p (the proposals).
struct LikPoint {
    bool init;
};

// The single-region way to evaluate one: the context's own kernels on its stream.
void enq_likelihood(Enq& q, const LikPoint& lp)
{
    spa_ctx* c = q.c;
    Workspace& w = c->ws;
    const bool mala = c->cfg.move_kind == SPA_MOVE_MALA;
    float* out = lp.init ? w.gl : w.gl_p;
    const float* src = lp.init ? w.beta : w.beta_p;
    if (mala && c->cfg.precision == SPA_PREC_SPLIT_BF16) {
        enq_grad_tc(q, out, src, 0.0, w.N);  // also leaves the softplus partials
        return;
    }
    enq_loglik(q);
    if (mala) {
        q.ck(launch_grad_simt(src, c->Xf, c->y, w.N, c->n, (int)c->p, w.eta, out, nullptr, c->pr, 0.0, q.st));
        ++q.launches;  // the plain adjoint is two kernels
    }
}

// One sweep of one context, enqueued piecewise: next() enqueues everything up to the sweep's
// next likelihood evaluation and stops there, so that a batch can evaluate the likelihoods of
// many regions' particles in one grouped launch before any region goes on. Between two
// stops the work is in the order of Section 4: init; then per scale step reweight,
// log-sum-exp / ESS, conditional resampling, proposal scales, M x (the MH test of the pending
// proposal fused with the next proposal, its likelihood), the last MH test with its commit,
// the summaries. A move's MH test runs at the start of the next move's proposal kernel.
class SweepGen {
public:
    SweepGen(spa_ctx* c, int64_t T, int M) : c_(c), T_(T), M_(M)
    {
        const spa_config& cfg = c->cfg;
        mala_ = cfg.move_kind == SPA_MOVE_MALA;
        site_ = cfg.move_kind == SPA_MOVE_SITE;
        // The step's summaries overlap the next step when that step is many short kernels
        // (RW, MALA). The single-coordinate cycle is one long launch per step whose blocks fill
        // the SMs: the summaries would only take SMs from it (measured 2% slower), so they stay
        // inline.
        fork_sum_ = !site_;
        // acceptance is per proposal: per coordinate update for the single-coordinate cycle
        denom_ = (double)c->ws.N * (double)M * (site_ ? (double)c->p : 1.0);
        sa_.nq = cfg.n_quantiles;
        sa_.nd = cfg.n_deltas;
        for (int k = 0; k < 8; ++k) {
            sa_.q[k] = cfg.quantiles[k];
            sa_.delta[k] = cfg.deltas[k];
        }
    }

    // Enqueue up to the next likelihood evaluation; true with *lp set if stopped at one (the
    // caller enqueues it, then calls next again), false when the sweep is complete.
    bool next(Enq& q, LikPoint* lp)
    {
        spa_ctx* c = c_;
        Workspace& w = c->ws;
        RunBufs& r = c->rb;
        const spa_config& cfg = c->cfg;
        const int p = (int)c->p;
        const WeightArrays wa{w.logw, w.W, w.Wf, w.wfix};
        for (;;) {
            switch (st_) {
            case START: {
                if (q.e == cudaSuccess) q.e = cudaMemsetAsync(r.acc, 0, sizeof(unsigned long long) * (size_t)(T_ + 1), q.st);
                if (q.e == cudaSuccess) q.e = cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), q.st);
                if (mala_) q.ck(launch_set_f64(w.lambda, cfg.mala_h, q.st));
                q.ck(launch_step_constants(c->pr, r.sched, (int)T_, p, r.stepk, r.rk, q.st));
                // t = 0: prior draws, their log-likelihoods, importance weights
                q.ck(launch_init_prior(w.beta, w.N, p, c->pr, r.sched, 0, r.seed, q.st));
                const MoveArgs a0 = move_args(c, nullptr);
                q.ck(launch_move_rw(a0, false, w.N, p, c->pr, r.stepk, 0, 0u, 0u, r.seed, 0, c->d_err, q.st));
                st_ = AFTER_INIT;
                lp->init = true;
                return true;
            }
            case AFTER_INIT: {
                q.ck(launch_finish_loglik(mh_state(c, nullptr), w.N, w.logw, nullptr, c->d_err, q.st));
                if (c->fault & FAULT_NAN_WEIGHT) q.ck(launch_set_f64(w.logw, std::nan(""), q.st));
                const bool rm = cfg.init_mode == SPA_INIT_RESAMPLE_MOVE;
                q.ck(launch_lse_ess(wa, w.N, w.lse_scratch, w.lse_counter, 0, rm ? 2 : 1, cfg.ess_frac, r.ess, r.logz,
                                    r.res, w.flag, c->d_err, q.st));
                ++q.launches;  // log-sum-exp is two kernels
                if (rm) {
                    enq_resample(q, 0);
                    b_ = 0;
                    st_ = BURN_BEGIN;
                } else {
                    t_ = 0;
                    st_ = STEP_BEGIN;
                }
                break;
            }
            case BURN_BEGIN: {
                if (b_ == cfg.burn_in_steps) {
                    q.ck(launch_mark_uniform(w.N, 0, r.ess, r.res, w.flag, q.st));
                    t_ = 0;
                    st_ = STEP_BEGIN;
                    break;
                }
                unsigned long long* scratch = r.acc + T_;
                if (q.e == cudaSuccess) q.e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), q.st);
                if (!site_) enq_colstats(q, 0);
                begin_moves(q, 0, m_base_, scratch, BURN_MOVE, BURN_END);
                break;
            }
            case BURN_END: {
                if (mala_) q.ck(launch_adapt_lambda(w.lambda, r.acc + T_, denom_, q.st));
                m_base_ += (uint32_t)M_;
                ++b_;
                st_ = BURN_BEGIN;
                break;
            }
            case STEP_BEGIN: {
                if (t_ == T_) {
                    // the last summaries
                    if (fork_sum_ && T_ > 0 && q.e == cudaSuccess) q.e = cudaStreamWaitEvent(q.st, c->ev_join, 0);
                    q.ck(launch_accept_rate(r.acc, (int)T_, denom_, r.accrate, q.st));
                    st_ = DONE;
                    break;
                }
                const int t = (int)t_;
                if (t > 0) {
                    q.ck(launch_reweight(w.beta, w.logw, w.lpq, w.N, p, c->pr, r.rk, t, c->d_err, q.st));
                    // the previous step's transpose has read beta and the weights (forked runs)
                    if (fork_sum_ && q.e == cudaSuccess) q.e = cudaStreamWaitEvent(q.st, c->ev_keys, 0);
                    q.ck(launch_lse_ess(wa, w.N, w.lse_scratch, w.lse_counter, t, 0, cfg.ess_frac, r.ess, r.logz, r.res,
                                        w.flag, c->d_err, q.st));
                    ++q.launches;
                }
                enq_resample(q, t);
                if (!site_) enq_colstats(q, t);
                begin_moves(q, t, t == 0 ? m_base_ : 0u, r.acc + t, STEP_MOVE, STEP_END);
                break;
            }
            case BURN_MOVE:
            case STEP_MOVE: {
                if (mm_ == M_) {
                    // the last MH test of the block, with the commit of its accepted rows
                    const MoveArgs a = move_args(c, acc_);
                    q.ck(launch_move_commit(a, mala_, w.N, p, c->pr, r.stepk, mt_, m0_ + (uint32_t)(M_ - 1), r.seed,
                                            c->d_err, q.st));
                    st_ = after_moves_;
                    break;
                }
                const MoveArgs a = move_args(c, acc_);
                const uint32_t m = m0_ + (uint32_t)mm_;
                if (mala_)
                    q.ck(launch_move_mala(a, mm_ > 0, w.N, p, c->pr, r.stepk, mt_, m, m - 1u, r.seed, c->d_err, q.st));
                else
                    q.ck(launch_move_rw(a, mm_ > 0, w.N, p, c->pr, r.stepk, mt_, m, m - 1u, r.seed, 1, c->d_err, q.st));
                ++mm_;
                lp->init = false;
                return true;
            }
            case STEP_END: {
                const int t = (int)t_;
                if (fork_sum_) {
                    // The key transpose and the summaries of step t run on the side stream beside
                    // step t + 1. The transpose reads beta and the weights, which step t + 1 first
                    // rewrites in its normalisation (it waits for ev_keys before); it copies the
                    // weights for the summaries, which then read nothing that the main stream writes.
                    if (q.e == cudaSuccess) q.e = cudaEventRecord(c->ev_fork, q.st);
                    if (q.e == cudaSuccess) q.e = cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0);
                    q.ck(launch_keys(w.beta, w.Wf, w.wfix, w.N, p, w.keysT, w.WfS, w.wfixS, false, c->side_stream));
                    if (q.e == cudaSuccess) q.e = cudaEventRecord(c->ev_keys, c->side_stream);
                    q.ck(launch_summaries_keys(w.keysT, w.WfS, w.wfixS, w.N, p, sa_, t, r.mean, r.quant, r.conc, false,
                                               c->side_stream));
                    if (q.e == cudaSuccess) q.e = cudaEventRecord(c->ev_join, c->side_stream);
                } else {
                    q.ck(launch_summaries(w.beta, w.Wf, w.wfix, w.N, p, sa_, t, r.mean, r.quant, r.conc, w.keysT, q.st));
                    ++q.launches;  // the key transpose and the summaries
                }
                if (cfg.map_path)
                    q.ck(launch_best_particle(mh_state(c, nullptr), w.beta, w.N, p, c->pr, r.sched, t, r.best, q.st));
                if (mala_) q.ck(launch_adapt_lambda(w.lambda, r.acc + t, denom_, q.st));
                ++t_;
                st_ = STEP_BEGIN;
                break;
            }
            case DONE:
                return false;
            }
        }
    }

private:
    enum Stage { START, AFTER_INIT, BURN_BEGIN, BURN_MOVE, BURN_END, STEP_BEGIN, STEP_MOVE, STEP_END, DONE };

    // M moves at step t with move indices m0 .. m0+M-1 (all M cycles in one launch for the
    // single-coordinate kernel, which needs no likelihood evaluations), then `after`.
    void begin_moves(Enq& q, int t, uint32_t m0, unsigned long long* acc, Stage moves, Stage after)
    {
        spa_ctx* c = c_;
        Workspace& w = c->ws;
        if (M_ <= 0) {
            st_ = after;
            return;
        }
        if (site_) {
            const float inv_sp = c->cfg.precision == SPA_PREC_SPLIT_BF16 ? (float)LOG2E : 1.0f;
            const SiteArgs sa{w.beta, w.llq, w.lpq, inv_sp, c->XT2, c->colf + c->p, (float)c->cfg.site_sd, acc};
            q.ck(launch_move_site(sa, w.N, (int)c->p, c->n, c->pr, c->rb.stepk, t, m0, M_, c->rb.seed, q.st));
            st_ = after;
            return;
        }
        mt_ = t;
        m0_ = m0;
        acc_ = acc;
        mm_ = 0;
        after_moves_ = after;
        st_ = moves;
    }

    spa_ctx* c_;
    int64_t T_;
    int M_;
    bool mala_ = false, site_ = false, fork_sum_ = true;
    double denom_ = 0.0;
    SummaryArgs sa_;
    Stage st_ = START;
    int64_t t_ = 0;
    int b_ = 0;
    uint32_t m_base_ = 0;
    // the current block of moves
    int mt_ = 0, mm_ = 0;
    uint32_t m0_ = 0;
    unsigned long long* acc_ = nullptr;
    Stage after_moves_ = STEP_END;
};

int64_t enqueue_sweep(spa_ctx* c, int64_t T, int M, cudaError_t* err_out)
{
    Enq q;
    q.c = c;
    q.st = c->stream();
    SweepGen gen(c, T, M);
    LikPoint lp;
    while (gen.next(q, &lp)) enq_likelihood(q, lp);
    *err_out = q.e;
    return q.launches;
}

int validate_config(spa_ctx* c, const spa_config& k)
{
    if (k.move_kind != SPA_MOVE_RW && k.move_kind != SPA_MOVE_MALA && k.move_kind != SPA_MOVE_SITE)
        return fail(c, SPA_EINVAL, "move_kind");
    if (k.move_kind == SPA_MOVE_SITE) {
        if (!(k.site_sd > 0.0) || !std::isfinite(k.site_sd)) return fail(c, SPA_EINVAL, "site_sd must be finite and > 0");
        if (c && site_warps_per_block(c->n, (int)c->p) < 1)
            return fail(c, SPA_EINVAL, "n + p too large for the single-coordinate kernel's shared memory");
    }
    if (k.precision != SPA_PREC_SPLIT_BF16 && k.precision != SPA_PREC_FP32) return fail(c, SPA_EINVAL, "precision");
    if (k.init_mode != SPA_INIT_PRIOR_IS && k.init_mode != SPA_INIT_RESAMPLE_MOVE) return fail(c, SPA_EINVAL, "init_mode");
    if (k.burn_in_steps < 0) return fail(c, SPA_EINVAL, "burn_in_steps");
    if (k.n_quantiles < 0 || k.n_quantiles > SPA_MAX_QUANTILES) return fail(c, SPA_EINVAL, "n_quantiles");
    for (int i = 0; i < k.n_quantiles; ++i)
        if (!(k.quantiles[i] > 0.0 && k.quantiles[i] < 1.0)) return fail(c, SPA_EINVAL, "quantile level");
    if (k.n_deltas < 0 || k.n_deltas > SPA_MAX_DELTAS) return fail(c, SPA_EINVAL, "n_deltas");
    for (int i = 0; i < k.n_deltas; ++i)
        if (!(k.deltas[i] > 0.0) || !std::isfinite(k.deltas[i])) return fail(c, SPA_EINVAL, "delta");
    if (!(k.ess_frac >= 0.0 && k.ess_frac <= 1.0)) return fail(c, SPA_EINVAL, "ess_frac");
    if (!(k.rw_scale > 0.0) || !(k.mala_h > 0.0) || !(k.sd_floor >= 0.0)) return fail(c, SPA_EINVAL, "scale parameters");
    return SPA_OK;
}

int upload_data(spa_ctx* c, const int8_t* G, const uint8_t* y)
{
    const int64_t n = c->n, p = c->p;
    cudaStream_t st = c->stream();
    CK(cudaMemcpyAsync(c->G, G, (size_t)(n * p), cudaMemcpyHostToDevice, st), "copy G");
    CK(cudaMemcpyAsync(c->y, y, (size_t)n, cudaMemcpyHostToDevice, st), "copy y");
    CK(cudaMemsetAsync(c->sums, 0, sizeof(unsigned long long) * (size_t)(3 * p + 1), st), "memset sums");
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), st), "memset err");
    CK(launch_store_sums(c->G, c->y, n, p, c->sums, c->d_err, st), "store sums");
    CK(launch_store_finish(c->G, n, p, c->Kp, c->sums, c->mean, c->sd, c->v, c->l2e_s, c->mean_f, c->colf, c->Gbf, c->Xf,
                           c->d_err, st),
       "store pack");
    CK(launch_store_pack_t(c->G, c->y, n, p, c->n_r, c->GT, c->yv, st), "store pack transposed");
    CK(launch_store_ybits(c->y, n, c->ywords, c->ybits, st), "store y bits");
    CK(launch_store_xt2(c->Xf, n, p, c->XT2, st), "store X transposed");
    c->lip_ok = false;  // new data: the MAP solver's curvature bound is recomputed on demand
    return read_error_word(c);
}

void destroy(spa_ctx* c)
{
    if (!c) return;
    drop_graph(c);
    free_workspace(c->ws);
    free_runbufs(c->rb);
    dfree(c->G); dfree(c->y); dfree(c->sums); dfree(c->mean); dfree(c->sd); dfree(c->v); dfree(c->unit_c); dfree(c->unit_k);
    dfree(c->l2e_s); dfree(c->mean_f); dfree(c->colf); dfree(c->Xf); dfree(c->Gbf); dfree(c->d_err); dfree(c->GT); dfree(c->yv);
    dfree(c->ybits); dfree(c->XT2); dfree(c->lip);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_keys) cudaEventDestroy(c->ev_keys);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->side_stream) cudaStreamDestroy(c->side_stream);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
}

}  // namespace

// ------------------------------------------------------------------ batches
// One grouped likelihood launch of a lock-step batch: the regions whose likelihood kernels
// share a tile class (n-tile width, resident particle operand), their table and the CTAs'
// unit ranges, in device memory.
struct BatchClass {
    int cfg = 0;
    bool ar = false;
    int R = 0;
    int grid = 0;
    TcRegion* regs = nullptr;
    int64_t* cta_units = nullptr;
};

struct spa_batch {
    std::vector<spa_ctx*> ctxs;
    std::vector<uint64_t> gens, seeds;
    std::vector<int64_t> T, per_ctx_launches;
    cudaStream_t st = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> joins;
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;
    // lock-step mode: every region stops at each likelihood evaluation, and one grouped launch
    // per tile class evaluates all regions' particles
    bool grouped = false;
    std::vector<BatchClass> classes;
    std::vector<cudaEvent_t> ev_lik;
    cudaEvent_t ev_grouped = nullptr;
    uint32_t* d_err = nullptr;  // the grouped launches' device error word
};

namespace {

void batch_free(spa_batch* b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (BatchClass& k : b->classes) {
        dfree(k.regs);
        dfree(k.cta_units);
    }
    dfree(b->d_err);
    for (cudaEvent_t ev : b->ev_lik)
        if (ev) cudaEventDestroy(ev);
    if (b->ev_grouped) cudaEventDestroy(b->ev_grouped);
    for (cudaEvent_t ev : b->joins)
        if (ev) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->st) cudaStreamDestroy(b->st);
    delete b;
}

// Lock-step batching (SPA_BATCH_MODE=lockstep) needs every region's sweep to stop at the
// same likelihood evaluations: the same T, N, M, move kind (random walk or MALA), start and
// burn-in, all on the tensor cores. By default the batch is one graph branch per region: on
// the 64-region batched workload that measures 1.84 s per batch against 2.26 s in lock step,
// whose joins at every evaluation stop the regions' other kernels from overlapping.
// The SMs each region's likelihood launches are sized for when a batch runs its regions as
// graph branches side by side: an eighth of the GPU once 8 or more regions share it, else
// an equal share. Smaller grids give each CTA more units (the per-CTA set-up and last
// epilogue are paid fewer times over the batch's work), while the other regions' branches
// keep the SMs busy. The likelihood partials are per 32 individuals whatever the grid, so
// the batch's results stay bit-identical to single runs.
int batch_plan_sms(int num_sms, int32_t R)
{
    const int share = R > 0 ? num_sms / (R < 8 ? R : 8) : num_sms;
    return share > 0 ? share : 1;
}

bool batch_lockstep(spa_ctx* const* ctxs, int32_t R, const spa_batch_args* args)
{
    const char* env = std::getenv("SPA_BATCH_MODE");
    if (!env || std::strcmp(env, "lockstep") != 0) return false;
    if (R < 2) return false;
    const spa_config& k0 = ctxs[0]->cfg;
    for (int32_t r = 0; r < R; ++r) {
        const spa_config& k = ctxs[r]->cfg;
        if (k.precision != SPA_PREC_SPLIT_BF16 || k.move_kind == SPA_MOVE_SITE) return false;
        if (k.move_kind != k0.move_kind || k.init_mode != k0.init_mode || k.burn_in_steps != k0.burn_in_steps)
            return false;
        if (args->T[r] != args->T[0] || args->N[r] != args->N[0] || args->moves_per_step[r] != args->moves_per_step[0])
            return false;
    }
    return true;
}

// The grouped launches' tables: regions by tile class, each class's units in region order,
// and CTA b's units [cta_units[b], cta_units[b + 1]) split by work (a unit of region r costs
// its kblocks_r k-blocks of the same 128 x BN tile).
int batch_build_classes(spa_batch* b)
{
    const int32_t R = (int32_t)b->ctxs.size();
    std::map<std::pair<int, bool>, std::vector<int32_t>> by_class;
    for (int32_t r = 0; r < R; ++r) {
        const TcPlan plan = plan_of(b->ctxs[r]);
        by_class[{plan.cfg, tc_plan_resident(plan)}].push_back(r);
    }
    const bool mala = b->ctxs[0]->cfg.move_kind == SPA_MOVE_MALA;
    for (const auto& kv : by_class) {
        BatchClass k;
        k.cfg = kv.first.first;
        k.ar = kv.first.second;
        k.R = (int)kv.second.size();
        std::vector<TcRegion> regs((size_t)k.R);
        std::vector<double> cum((size_t)k.R + 1, 0.0);
        int64_t units = 0;
        for (int i = 0; i < k.R; ++i) {
            spa_ctx* c = b->ctxs[kv.second[(size_t)i]];
            const Workspace& w = c->ws;
            const TcPlan plan = plan_of(c);
            TcRegion& g = regs[(size_t)i];
            std::memset(&g, 0, sizeof(g));
            g.A = w.mapA;
            g.At = plan.tw ? w.mapAt : w.mapA;
            g.B = c->mapB;
            g.Bt = plan.tw ? c->mapBt : c->mapB;
            g.partial = w.partial;
            g.ybits = c->ybits;
            if (mala) {
                const AdjPlan a = adj_plan((int)c->p, c->n, w.N_pad, c->num_sms);
                g.R = w.R;
                g.n_r = a.n_r;
                g.rsum_part = w.rsum;
            }
            g.N_pad = w.N_pad;
            g.unit0 = units;
            g.tw = plan.tw;
            g.n_tiles = plan.n_tiles;
            g.m_tiles = plan.m_tiles;
            g.kblocks = plan.kblocks;
            g.ksteps = plan.ksteps;
            g.Kp = c->Kp;
            g.n = (int)c->n;
            const int64_t u_r = (int64_t)plan.m_tiles * plan.n_tiles;
            units += u_r;
            cum[(size_t)i + 1] = cum[(size_t)i] + (double)u_r * plan.kblocks;
        }
        const int num_sms = b->ctxs[0]->num_sms;
        k.grid = (int)std::min<int64_t>(units, num_sms);
        std::vector<int64_t> cu((size_t)k.grid + 1);
        int i = 0;
        for (int cb = 0; cb <= k.grid; ++cb) {
            const double target = cum[(size_t)k.R] * cb / k.grid;
            while (i < k.R - 1 && cum[(size_t)i + 1] <= target) ++i;
            const double inside = (target - cum[(size_t)i]) / regs[(size_t)i].kblocks;
            int64_t u = regs[(size_t)i].unit0 + (int64_t)std::ceil(inside - 1e-9);
            if (cb == k.grid) u = units;
            if (cb > 0 && u < cu[(size_t)cb - 1]) u = cu[(size_t)cb - 1];
            cu[(size_t)cb] = u < units ? u : units;
        }
        cudaError_t e = dalloc(&k.regs, regs.size());
        if (e == cudaSuccess) e = dalloc(&k.cta_units, cu.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(k.regs, regs.data(), sizeof(TcRegion) * regs.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(k.cta_units, cu.data(), sizeof(int64_t) * cu.size(), cudaMemcpyHostToDevice);
        b->classes.push_back(k);
        if (e != cudaSuccess) {
            set_thread_error_str(std::string("batch: grouped tables: ") + cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? SPA_ENOMEM : SPA_ECUDA;
        }
    }
    return SPA_OK;
}

// Capture of a lock-step batch: each region's sweep runs on its own stream up to its next
// likelihood evaluation; then the batch stream waits for all of them, one grouped launch per
// tile class evaluates every region's packed particles (in the residual mode on the MALA
// path), and each region goes on after it (with its adjoint and gradient on the MALA path).
cudaError_t batch_capture_lockstep(spa_batch* b, const spa_batch_args* args)
{
    const int32_t R = (int32_t)b->ctxs.size();
    const bool mala = b->ctxs[0]->cfg.move_kind == SPA_MOVE_MALA;
    const uint64_t wait_ns = b->ctxs[0]->wait_ns;
    std::vector<SweepGen> gens;
    std::vector<Enq> qs((size_t)R);
    gens.reserve((size_t)R);
    for (int32_t r = 0; r < R; ++r) {
        gens.emplace_back(b->ctxs[r], b->T[r], args->moves_per_step[r]);
        qs[(size_t)r].c = b->ctxs[r];
        qs[(size_t)r].st = b->ctxs[r]->stream();
    }
    cudaError_t e = cudaSuccess;
    for (;;) {
        int stopped = 0;
        LikPoint lp{};
        for (int32_t r = 0; r < R; ++r) {
            LikPoint l{};
            if (gens[(size_t)r].next(qs[(size_t)r], &l)) {
                ++stopped;
                lp = l;
            }
            if (qs[(size_t)r].e != cudaSuccess) return qs[(size_t)r].e;
        }
        if (stopped == 0) break;
        if (stopped != R) return cudaErrorInvalidValue;  // the regions' sweeps are not in lock step
        for (int32_t r = 0; r < R && e == cudaSuccess; ++r) {
            e = cudaEventRecord(b->ev_lik[(size_t)r], qs[(size_t)r].st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->ev_lik[(size_t)r], 0);
        }
        for (const BatchClass& k : b->classes) {
            if (e == cudaSuccess)
                e = launch_loglik_tc_grouped(k.regs, k.R, k.cta_units, k.grid, k.cfg, k.ar, mala, b->d_err, b->st,
                                             wait_ns);
            ++b->launches;
        }
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_grouped, b->st);
        for (int32_t r = 0; r < R && e == cudaSuccess; ++r) {
            e = cudaStreamWaitEvent(qs[(size_t)r].st, b->ev_grouped, 0);
            if (e == cudaSuccess && mala) {
                Workspace& w = b->ctxs[r]->ws;
                enq_grad_tail(qs[(size_t)r], lp.init ? w.gl : w.gl_p, lp.init ? w.beta : w.beta_p, 0.0, w.N);
                e = qs[(size_t)r].e;
            }
        }
        if (e != cudaSuccess) return e;
    }
    for (int32_t r = 0; r < R; ++r) {
        b->per_ctx_launches.push_back(qs[(size_t)r].launches);
        b->launches += qs[(size_t)r].launches;
        if (e == cudaSuccess) e = cudaEventRecord(b->joins[(size_t)r], qs[(size_t)r].st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->joins[(size_t)r], 0);
    }
    return e;
}

// Prepare every context (buffers, schedule, seed), then capture all sweeps into one graph:
// the batch stream forks to each context's stream, each context enqueues its sweep there,
// and the batch stream joins them all.
int batch_build(spa_batch* b, spa_ctx* const* ctxs, int32_t R, const spa_batch_args* args)
{
    for (int32_t r = 0; r < R; ++r) {
        spa_ctx* c = ctxs[r];
        const int64_t T = args->T[r], N = args->N[r];
        const int32_t M = args->moves_per_step[r];
        const double* sched = args->schedules[r];
        auto bad = [&](const char* what) {
            set_thread_error_str("region " + std::to_string(r) + ": " + what);
            return SPA_EINVAL;
        };
        if (!sched) return bad("schedule is NULL");
        if (T < 1 || T > (int64_t)1 << 24) return bad("T out of range");
        if (N < 1 || N > (int64_t)1 << 22) return bad("N out of range");
        if (M < 0 || M > 65535) return bad("moves_per_step out of range");
        for (int64_t t = 0; t < T; ++t)
            if (!(sched[t] > 0.0) || !std::isfinite(sched[t])) return bad("schedule values must be finite and > 0");
        int rc = validate_config(c, c->cfg);
        if (rc == SPA_OK) rc = ensure_workspace(c, N);
        if (rc == SPA_OK) rc = ensure_runbufs(c, T);
        if (rc == SPA_OK && c->cfg.move_kind == SPA_MOVE_MALA) rc = ensure_mala_buffers(c);
        if (rc == SPA_OK) {
            cudaError_t e = cudaMemcpyAsync(c->rb.sched, sched, sizeof(double) * (size_t)T, cudaMemcpyHostToDevice,
                                            c->stream());
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream());
            if (e != cudaSuccess) rc = cuda_fail(c, e, "copy schedule");
        }
        if (rc != SPA_OK) {
            set_thread_error_str("region " + std::to_string(r) + ": " + c->err);
            return rc;
        }
        b->ctxs.push_back(c);
        b->T.push_back(T);
        b->seeds.push_back(args->seeds[r]);
    }
    auto cuda_err = [&](cudaError_t e, const char* what) {
        set_thread_error_str(std::string("batch: ") + what + ": " + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SPA_ENOMEM : SPA_ECUDA;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    b->joins.assign((size_t)R, nullptr);
    for (int32_t r = 0; r < R && e == cudaSuccess; ++r) e = cudaEventCreateWithFlags(&b->joins[r], cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_err(e, "stream and events");
    b->grouped = batch_lockstep(ctxs, R, args);
    if (b->grouped) {
        b->ev_lik.assign((size_t)R, nullptr);
        for (int32_t r = 0; r < R && e == cudaSuccess; ++r)
            e = cudaEventCreateWithFlags(&b->ev_lik[(size_t)r], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_grouped, cudaEventDisableTiming);
        if (e == cudaSuccess) e = dalloc(&b->d_err, 1);
        if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(uint32_t));
        if (e != cudaSuccess) return cuda_err(e, "lock-step events");
        const int rc = batch_build_classes(b);
        if (rc != SPA_OK) return rc;
    }
    e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_err(e, "begin capture");
    cudaError_t ee = cudaEventRecord(b->fork, b->st);
    b->launches = 0;
    if (b->grouped) {
        for (int32_t r = 0; r < R && ee == cudaSuccess; ++r) ee = cudaStreamWaitEvent(b->ctxs[r]->stream(), b->fork, 0);
        if (ee == cudaSuccess) ee = batch_capture_lockstep(b, args);
    } else {
        for (int32_t r = 0; r < R && ee == cudaSuccess; ++r) {
            spa_ctx* c = b->ctxs[r];
            ee = cudaStreamWaitEvent(c->stream(), b->fork, 0);
            if (ee != cudaSuccess) break;
            c->plan_sms = batch_plan_sms(c->num_sms, R);  // only while this batch's graph is captured
            const int64_t n = enqueue_sweep(c, b->T[r], args->moves_per_step[r], &ee);
            c->plan_sms = 0;
            b->per_ctx_launches.push_back(n);
            b->launches += n;
            if (ee == cudaSuccess) ee = cudaEventRecord(b->joins[r], c->stream());
            if (ee == cudaSuccess) ee = cudaStreamWaitEvent(b->st, b->joins[r], 0);
        }
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->st, &g);
    if (ee != cudaSuccess || ec != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_err(ee != cudaSuccess ? ee : ec, "capture");
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return cuda_err(e, "graph instantiate");
    }
    for (int32_t r = 0; r < R; ++r) b->gens.push_back(b->ctxs[r]->gen);
    return SPA_OK;
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

void spa_config_default(spa_config* k)
{
    if (!k) return;
    std::memset(k, 0, sizeof(*k));
    k->move_kind = SPA_MOVE_RW;
    k->precision = SPA_PREC_SPLIT_BF16;
    k->init_mode = SPA_INIT_PRIOR_IS;
    k->burn_in_steps = 0;
    k->n_quantiles = 3;
    k->quantiles[0] = 0.05;
    k->quantiles[1] = 0.5;
    k->quantiles[2] = 0.95;
    k->n_deltas = 2;
    k->deltas[0] = 0.05;
    k->deltas[1] = 0.1;
    k->ess_frac = 0.75;
    k->rw_scale = 2.38;
    k->mala_h = 1.65;
    k->sd_floor = 1e-3;
    k->site_sd = 0.5;
    k->map_path = 0;
    k->stream = nullptr;
}

int spa_create(const int8_t* G, const uint8_t* y, int64_t n, int64_t p, double nu, spa_ctx** out)
{
    if (!out) return fail(nullptr, SPA_EINVAL, "out is NULL");
    *out = nullptr;
    if (!G || !y) return fail(nullptr, SPA_EINVAL, "G or y is NULL");
    if (n < 1 || p < 1 || n > (int64_t)1 << 24 || p > 8192) return fail(nullptr, SPA_EINVAL, "n or p out of range");
    if (!(nu > 0.0)) return fail(nullptr, SPA_EINVAL, "nu must be > 0 (or +INFINITY)");
    spa_ctx* c = new (std::nothrow) spa_ctx();
    if (!c) return fail(nullptr, SPA_ENOMEM, "host allocation");
    int rc = check_device(c);
    if (rc != SPA_OK) {
        set_thread_error_str(c->err);
        destroy(c);
        return rc;
    }
    spa_config_default(&c->cfg);
    c->n = n;
    c->p = p;
    c->Kp = (int)round_up(p + 1, 64);
    c->nu = nu;
    c->pr.de = std::isinf(nu) ? 1 : 0;
    c->pr.a = c->pr.de ? 1.0f : (float)nu;
    cudaError_t e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_keys, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
#define CA(ptr, cnt) \
    if (e == cudaSuccess) e = dalloc(&c->ptr, (size_t)(cnt))
    CA(G, n * p);
    CA(y, n);
    CA(sums, 3 * p + 1);
    CA(mean, p); CA(sd, p); CA(v, p); CA(unit_c, 1); CA(unit_k, 1);
    CA(l2e_s, p); CA(mean_f, p); CA(colf, 3 * p);
    CA(Xf, n * p);
    CA(Gbf, n * c->Kp);
    c->n_r = round_up(n, 64);
    CA(GT, p * c->n_r);
    CA(yv, n);
    CA(XT2, n * p);
    CA(lip, 1);
    c->ywords = round_up(n, 256) / 32;
    CA(ybits, c->ywords);
    CA(d_err, 1);
#undef CA
    if (e != cudaSuccess) {
        set_thread_error_str(std::string("device allocation: ") + cudaGetErrorString(e));
        destroy(c);
        return e == cudaErrorMemoryAllocation ? SPA_ENOMEM : SPA_ECUDA;
    }
    const double one = 1.0;
    e = cudaMemcpy(c->unit_c, &one, sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_step_constants(c->pr, c->unit_c, 1, (int)c->p, c->unit_k, nullptr, c->own_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->own_stream);
    if (e != cudaSuccess) {
        set_thread_error_str(cudaGetErrorString(e));
        destroy(c);
        return SPA_ECUDA;
    }
    rc = upload_data(c, G, y);
    if (rc != SPA_OK) {
        set_thread_error_str(c->err);
        destroy(c);
        return rc;
    }
    *out = c;
    return SPA_OK;
}

int spa_set_data(spa_ctx* c, const int8_t* G, const uint8_t* y)
{
    if (!c) return fail(nullptr, SPA_EINVAL, "ctx is NULL");
    if (!G || !y) return fail(c, SPA_EINVAL, "G or y is NULL");
    return upload_data(c, G, y);
}

int spa_set_config(spa_ctx* c, const spa_config* k)
{
    if (!c || !k) return fail(c, SPA_EINVAL, "NULL argument");
    int rc = validate_config(c, *k);
    if (rc != SPA_OK) return rc;
    if (std::memcmp(&c->cfg, k, sizeof(spa_config)) != 0) drop_graph(c);
    c->cfg = *k;
    return SPA_OK;
}

int spa_get_config(const spa_ctx* c, spa_config* k)
{
    if (!c || !k) return fail(nullptr, SPA_EINVAL, "NULL argument");
    *k = c->cfg;
    return SPA_OK;
}

void spa_destroy(spa_ctx* c) { destroy(c); }

const char* spa_last_error(const spa_ctx* c)
{
    if (c) return c->err.c_str();
    return g_thread_error;
}

int64_t spa_last_launch_count(const spa_ctx* c) { return c ? c->last_launches : 0; }

int spa_set_wait_limit(spa_ctx* c, uint64_t limit_ns)
{
    if (!c) return fail(nullptr, SPA_EINVAL, "ctx is NULL");
    if (limit_ns != c->wait_ns) drop_graph(c);  // the limit is a kernel argument of the captured sweep
    c->wait_ns = limit_ns;
    return SPA_OK;
}

int spa_loglik_tile_width(const spa_ctx* c) { return (c && c->ws.N > 0) ? c->ws.BN : 0; }

int spa_loglik_tile_config(const spa_ctx* c, int32_t* source)
{
    if (!c || c->ws.N <= 0) return -1;
    if (source) *source = c->ws.cfg_source;
    return c->ws.cfg;
}

int spa_set_tile_config(spa_ctx* c, int32_t cfg)
{
    if (!c) return fail(nullptr, SPA_EINVAL, "ctx is NULL");
    if (cfg < -1 || cfg >= TC_CONFIGS) return fail(c, SPA_EINVAL, "tile configuration out of range");
    if (cfg == c->tile_cfg) return SPA_OK;
    c->tile_cfg = cfg;
    drop_graph(c);
    free_workspace(c->ws);  // the next call builds the workspace with the new configuration
    return SPA_OK;
}

static int run_common(spa_ctx* c, const double* sched, bool sched_on_device, int64_t T, int64_t N, int32_t M,
                      uint64_t seed)
{
    if (!c) return fail(nullptr, SPA_EINVAL, "ctx is NULL");
    if (!sched) return fail(c, SPA_EINVAL, "schedule is NULL");
    if (T < 1 || T > (int64_t)1 << 24) return fail(c, SPA_EINVAL, "T out of range");
    if (N < 1 || N > (int64_t)1 << 22) return fail(c, SPA_EINVAL, "N out of range");
    if (M < 0 || M > 65535) return fail(c, SPA_EINVAL, "moves_per_step out of range");
    if (!sched_on_device)
        for (int64_t t = 0; t < T; ++t)
            if (!(sched[t] > 0.0) || !std::isfinite(sched[t])) return fail(c, SPA_EINVAL, "schedule values must be finite and > 0");
    int rc = validate_config(c, c->cfg);
    if (rc != SPA_OK) return rc;
    rc = ensure_workspace(c, N);
    if (rc != SPA_OK) return rc;
    rc = ensure_runbufs(c, T);
    if (rc != SPA_OK) return rc;
    if (c->cfg.move_kind == SPA_MOVE_MALA) {
        rc = ensure_mala_buffers(c);
        if (rc != SPA_OK) return rc;
    }
    cudaStream_t st = c->stream();
    CK(cudaMemcpyAsync(c->rb.sched, sched, sizeof(double) * (size_t)T,
                       sched_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st),
       "copy schedule");
    CK(cudaMemcpyAsync(c->rb.seed, &seed, sizeof(uint64_t), cudaMemcpyHostToDevice, st), "copy seed");
    GraphKey key;
    key.T = T;
    key.N = N;
    key.M = M;
    key.cfg = c->cfg;
    key.fault = fault_mask() & (FAULT_NAN_WEIGHT | FAULT_STALL);
    c->fault = key.fault;
    if (!c->gexec || !(key == c->gkey)) {
        drop_graph(c, false);  // buffers and config were settled above
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t ee = cudaSuccess;
        const int64_t launches = enqueue_sweep(c, T, M, &ee);
        cudaError_t ec = cudaStreamEndCapture(st, &g);
        if (ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(c, ee, "enqueue sweep");
        }
        if (ec != cudaSuccess) return cuda_fail(c, ec, "end capture");
        cudaError_t ei = cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            c->gexec = nullptr;
            return cuda_fail(c, ei, "graph instantiate");
        }
        c->gkey = key;
        c->graph_launches = launches;
    }
    CK(cudaGraphLaunch(c->gexec, st), "graph launch");
    c->last_launches = c->graph_launches;
    c->best_T = c->cfg.map_path ? T : 0;
    return SPA_OK;
}

int spa_run(spa_ctx* c, const double* sched, int64_t T, int64_t N, int32_t M, uint64_t seed, spa_result* out)
{
    int rc = run_common(c, sched, false, T, N, M, seed);
    if (rc != SPA_OK) return rc;
    cudaStream_t st = c->stream();
    const int64_t p = c->p;
    const int nq = c->cfg.n_quantiles, nd = c->cfg.n_deltas;
    if (out) {
        RunBufs& r = c->rb;
        auto d2h = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
            return dst ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st) : cudaSuccess;
        };
        CK(d2h(out->mean, r.mean, sizeof(double) * (size_t)(T * p)), "copy mean");
        CK(d2h(out->quantile, r.quant, sizeof(double) * (size_t)(T * p * nq)), "copy quantiles");
        CK(d2h(out->conc, r.conc, sizeof(double) * (size_t)(T * p * nd)), "copy concentrations");
        CK(d2h(out->ess, r.ess, sizeof(double) * (size_t)T), "copy ess");
        CK(d2h(out->log_z_inc, r.logz, sizeof(double) * (size_t)T), "copy log z");
        CK(d2h(out->accept_rate, r.accrate, sizeof(double) * (size_t)T), "copy acceptance");
        CK(d2h(out->resampled, r.res, (size_t)T), "copy resampled");
    }
    return read_error_word(c);
}

int spa_run_device(spa_ctx* c, const double* sched, int64_t T, int64_t N, int32_t M, uint64_t seed, spa_result* out)
{
    int rc = run_common(c, sched, true, T, N, M, seed);
    if (rc != SPA_OK) return rc;
    if (out) {
        cudaStream_t st = c->stream();
        const int64_t p = c->p;
        const int nq = c->cfg.n_quantiles, nd = c->cfg.n_deltas;
        RunBufs& r = c->rb;
        auto d2d = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
            return dst ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st) : cudaSuccess;
        };
        CK(d2d(out->mean, r.mean, sizeof(double) * (size_t)(T * p)), "copy mean");
        CK(d2d(out->quantile, r.quant, sizeof(double) * (size_t)(T * p * nq)), "copy quantiles");
        CK(d2d(out->conc, r.conc, sizeof(double) * (size_t)(T * p * nd)), "copy concentrations");
        CK(d2d(out->ess, r.ess, sizeof(double) * (size_t)T), "copy ess");
        CK(d2d(out->log_z_inc, r.logz, sizeof(double) * (size_t)T), "copy log z");
        CK(d2d(out->accept_rate, r.accrate, sizeof(double) * (size_t)T), "copy acceptance");
        CK(d2d(out->resampled, r.res, (size_t)T), "copy resampled");
    }
    return SPA_OK;
}

int spa_sync(spa_ctx* c)
{
    if (!c) return fail(nullptr, SPA_EINVAL, "ctx is NULL");
    return read_error_word(c);
}

int spa_batch_create(spa_ctx* const* ctxs, int32_t R, const spa_batch_args* args, spa_batch** out)
{
    if (!out) return fail(nullptr, SPA_EINVAL, "out is NULL");
    *out = nullptr;
    if (!ctxs || !args || R < 1 || !args->schedules || !args->T || !args->N || !args->moves_per_step || !args->seeds)
        return fail(nullptr, SPA_EINVAL, "bad batch arguments");
    for (int32_t r = 0; r < R; ++r) {
        if (!ctxs[r]) return fail(nullptr, SPA_EINVAL, "NULL context in batch");
        for (int32_t q = 0; q < r; ++q)
            if (ctxs[q] == ctxs[r]) return fail(nullptr, SPA_EINVAL, "a context appears twice in the batch");
    }
    spa_batch* b = new (std::nothrow) spa_batch();
    if (!b) return fail(nullptr, SPA_ENOMEM, "host allocation");
    int rc = batch_build(b, ctxs, R, args);
    if (rc != SPA_OK) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return SPA_OK;
}

int spa_batch_run(spa_batch* b, const uint64_t* seeds, spa_result* outs)
{
    if (!b || !b->exec) return fail(nullptr, SPA_EINVAL, "batch is NULL");
    const int32_t R = (int32_t)b->ctxs.size();
    for (int32_t r = 0; r < R; ++r)
        if (b->ctxs[r]->gen != b->gens[r])
            return fail(nullptr, SPA_EINVAL, "a context's workspace or config changed since the batch was created");
    if (seeds)
        for (int32_t r = 0; r < R; ++r) b->seeds[r] = seeds[r];
    cudaStream_t st = b->st;
    cudaError_t e = cudaSuccess;
    if (b->d_err) e = cudaMemsetAsync(b->d_err, 0, sizeof(uint32_t), st);
    for (int32_t r = 0; r < R && e == cudaSuccess; ++r)
        e = cudaMemcpyAsync(b->ctxs[r]->rb.seed, &b->seeds[r], sizeof(uint64_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, st);
    for (int32_t r = 0; r < R && e == cudaSuccess && outs; ++r) {
        spa_ctx* c = b->ctxs[r];
        const RunBufs& rb = c->rb;
        const int64_t T = b->T[r], p = c->p;
        const int nq = c->cfg.n_quantiles, nd = c->cfg.n_deltas;
        spa_result* o = &outs[r];
        auto d2h = [&](void* dst, const void* src, size_t bytes) {
            if (dst && e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st);
        };
        d2h(o->mean, rb.mean, sizeof(double) * (size_t)(T * p));
        d2h(o->quantile, rb.quant, sizeof(double) * (size_t)(T * p * nq));
        d2h(o->conc, rb.conc, sizeof(double) * (size_t)(T * p * nd));
        d2h(o->ess, rb.ess, sizeof(double) * (size_t)T);
        d2h(o->log_z_inc, rb.logz, sizeof(double) * (size_t)T);
        d2h(o->accept_rate, rb.accrate, sizeof(double) * (size_t)T);
        d2h(o->resampled, rb.res, (size_t)T);
    }
    uint32_t grouped_err = 0;
    if (b->d_err && e == cudaSuccess)
        e = cudaMemcpyAsync(&grouped_err, b->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(nullptr, e == cudaErrorMemoryAllocation ? SPA_ENOMEM : SPA_ECUDA,
                                      std::string("batch run: ") + cudaGetErrorString(e));
    if (grouped_err) {
        const int rc = map_device_error(nullptr, grouped_err);
        set_thread_error_str(std::string("grouped likelihood launches: ") + g_thread_error);
        return rc;
    }
    for (int32_t r = 0; r < R; ++r) {
        spa_ctx* c = b->ctxs[r];
        c->last_launches = b->per_ctx_launches[r];
        c->best_T = c->cfg.map_path ? b->T[r] : 0;
        const int rc = read_error_word(c);
        if (rc != SPA_OK) {
            set_thread_error_str("region " + std::to_string(r) + ": " + c->err);
            return rc;
        }
    }
    return SPA_OK;
}

int64_t spa_batch_launch_count(const spa_batch* b) { return b ? b->launches : 0; }

void spa_batch_destroy(spa_batch* b) { batch_free(b); }

int spa_run_batch(spa_ctx* const* ctxs, int32_t R, const spa_batch_args* args, spa_result* outs)
{
    if (R == 0 && ctxs && args) return SPA_OK;
    spa_batch* b = nullptr;
    int rc = spa_batch_create(ctxs, R, args, &b);
    if (rc != SPA_OK) return rc;
    rc = spa_batch_run(b, nullptr, outs);
    spa_batch_destroy(b);
    return rc;
}

// ------------------------------------------------------------ per-step entry points
static int loglik_impl(spa_ctx* c, const float* B, bool B_dev, int64_t N, double* ll, bool ll_dev, cudaStream_t st_user)
{
    if (!c) return fail(nullptr, SPA_EINVAL, "ctx is NULL");
    if (!B || !ll || N < 1 || N > (int64_t)1 << 22) return fail(c, SPA_EINVAL, "bad arguments");
    int rc = ensure_workspace(c, N);
    if (rc != SPA_OK) return rc;
    cudaStream_t st = st_user ? st_user : c->stream();
    Workspace& w = c->ws;
    const int64_t p = c->p;
    const bool tc = c->cfg.precision == SPA_PREC_SPLIT_BF16;
    if (st_user) CK(cudaStreamSynchronize(c->stream()), "sync context stream");
    CK(cudaMemcpyAsync(w.beta, B, sizeof(float) * (size_t)(N * p), B_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       st),
       "copy B");
    const MoveArgs a = move_args(c, nullptr);
    CK(launch_move_rw(a, false, N, (int)p, c->pr, c->unit_k, 0, 0u, 0u, nullptr, 0, c->d_err, st), "pack");
    if (tc) {
        CK(launch_loglik_tc(maps_of(c), plan_of(c), c->n, c->Kp, c->ybits, w.partial, w.N_pad, c->d_err, st, nullptr,
                            c->wait_ns, fault_mask() & FAULT_STALL),
           "loglik tc");
    } else {
        CK(launch_loglik_simt(w.beta_p, c->Xf, c->y, N, c->n, (int)p, w.partial, w.N_pad, st), "loglik simt");
    }
    CK(launch_finish_loglik(a.mh, N, nullptr, ll_dev ? ll : w.ll, c->d_err, st), "finish loglik");
    if (!ll_dev) CK(cudaMemcpyAsync(ll, w.ll, sizeof(double) * (size_t)N, cudaMemcpyDeviceToHost, st), "copy ll");
    if (st != c->stream()) CK(cudaStreamSynchronize(st), "sync");
    return read_error_word(c);
}

int spa_loglik_repeat(spa_ctx* c, int64_t N, int32_t reps, void* stream)
{
    if (!c) return fail(nullptr, SPA_EINVAL, "ctx is NULL");
    if (c->ws.N != N || N < 1 || reps < 0) return fail(c, SPA_EINVAL, "no workspace of N particles");
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : c->stream();
    Workspace& w = c->ws;
    for (int32_t k = 0; k < reps; ++k) {
        if (c->cfg.precision == SPA_PREC_SPLIT_BF16) {
            CK(launch_loglik_tc(maps_of(c), plan_of(c), c->n, c->Kp, c->ybits, w.partial, w.N_pad, c->d_err, st, nullptr,
                            c->wait_ns),
               "loglik tc");
        } else {
            CK(launch_loglik_simt(w.beta_p, c->Xf, c->y, N, c->n, (int)c->p, w.partial, w.N_pad, st), "loglik simt");
        }
    }
    return SPA_OK;
}

int spa_grad_repeat(spa_ctx* c, int64_t N, int32_t reps, void* stream)
{
    if (!c) return fail(nullptr, SPA_EINVAL, "ctx is NULL");
    if (c->ws.N != N || N < 1 || reps < 0) return fail(c, SPA_EINVAL, "no workspace of N particles");
    if (c->cfg.precision != SPA_PREC_SPLIT_BF16 || c->cfg.move_kind != SPA_MOVE_MALA || !c->ws.R)
        return fail(c, SPA_EINVAL, "no split-BF16 MALA workspace (run a MALA sweep of N particles first)");
    Enq q;
    q.c = c;
    q.st = stream ? static_cast<cudaStream_t>(stream) : c->stream();
    Workspace& w = c->ws;
    for (int32_t k = 0; k < reps && q.e == cudaSuccess; ++k) enq_grad_tc(q, w.gl_p, w.beta_p, 0.0, w.N);
    if (q.e != cudaSuccess) return cuda_fail(c, q.e, "gradient kernels");
    return SPA_OK;
}

static MapData map_data(spa_ctx* c)
{
    return MapData{c->Xf, c->XT2, c->y, c->n, (int)c->p, c->lip, c->pr};
}

static int ensure_lipschitz(spa_ctx* c, cudaStream_t st)
{
    if (c->lip_ok) return SPA_OK;
    CK(launch_map_lipschitz(map_data(c), c->lip, st), "MAP curvature bound");
    CK(cudaStreamSynchronize(st), "sync");
    c->lip_ok = true;
    return SPA_OK;
}

int spa_map(spa_ctx* c, const float* beta0, int32_t S, double cs, int32_t max_em, double tol, float* beta_out,
            double* logpost)
{
    if (!c) return fail(nullptr, SPA_EINVAL, "ctx is NULL");
    if (!beta0 || !beta_out || S < 1 || !(cs > 0.0) || !std::isfinite(cs) || max_em < 1 || !(tol > 0.0))
        return fail(c, SPA_EINVAL, "bad arguments");
    if (!map_fits(c->n, (int)c->p)) return fail(c, SPA_EINVAL, "n + 5p too large for the MAP solver's shared memory");
    cudaStream_t st = c->stream();
    int rc = ensure_lipschitz(c, st);
    if (rc != SPA_OK) return rc;
    const int64_t p = c->p;
    float *d0 = nullptr, *d1 = nullptr;
    double* dl = nullptr;
    cudaError_t e = dalloc(&d0, (size_t)(S * p));
    if (e == cudaSuccess) e = dalloc(&d1, (size_t)(S * p));
    if (e == cudaSuccess) e = dalloc(&dl, (size_t)S);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d0, beta0, sizeof(float) * (size_t)(S * p), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_map(map_data(c), d0, S, cs, max_em, (float)tol, d1, dl, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(beta_out, d1, sizeof(float) * (size_t)(S * p), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && logpost) e = cudaMemcpyAsync(logpost, dl, sizeof(double) * (size_t)S, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(d0);
    dfree(d1);
    dfree(dl);
    if (e != cudaSuccess) return cuda_fail(c, e, "MAP");
    return read_error_word(c);
}

// The MAP path rounds from device arrays of starts best [T][p] and scales sched [T].
static int map_path_impl(spa_ctx* c, const float* best, const double* sched, int64_t T, int32_t max_em, double tol,
                         float* map_out, double* logpost)
{
    cudaStream_t st = c->stream();
    int rc = ensure_lipschitz(c, st);
    if (rc != SPA_OK) return rc;
    const int64_t p = c->p;
    MapRoundBufs b{};
    cudaError_t e = dalloc(&b.A, (size_t)(T * p));
    if (e == cudaSuccess) e = dalloc(&b.lpA, (size_t)T);
    if (e == cudaSuccess) e = dalloc(&b.S, (size_t)(2 * T * p));
    if (e == cudaSuccess) e = dalloc(&b.lpS, (size_t)(2 * T));
    if (e == cudaSuccess) e = dalloc(&b.chg, (size_t)(2 * T));
    if (e == cudaSuccess) e = dalloc(&b.n_changed, 1);
    // Round k leaves the first k + 1 steps final, so at most T rounds after round 0 change
    // anything; the loop ends at the first round that changes nothing.
    int last = 0;  // the last round launched; its copy holds the result
    if (e == cudaSuccess) e = launch_map_round(map_data(c), best, sched, (int)T, 0, max_em, (float)tol, b, st);
    for (int round = 1; e == cudaSuccess && round <= T; ++round) {
        int changed = 0;
        e = cudaMemsetAsync(b.n_changed, 0, sizeof(int), st);
        if (e == cudaSuccess) e = launch_map_round(map_data(c), best, sched, (int)T, round, max_em, (float)tol, b, st);
        if (e == cudaSuccess) last = round;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&changed, b.n_changed, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && changed == 0) break;
    }
    c->map_rounds = last;
    const int w = last & 1;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(map_out, b.S + w * T * p, sizeof(float) * (size_t)(T * p), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && logpost)
        e = cudaMemcpyAsync(logpost, b.lpS + w * T, sizeof(double) * (size_t)T, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(b.A);
    dfree(b.lpA);
    dfree(b.S);
    dfree(b.lpS);
    dfree(b.chg);
    dfree(b.n_changed);
    if (e != cudaSuccess) return cuda_fail(c, e, "MAP path");
    return read_error_word(c);
}

int spa_map_path(spa_ctx* c, int64_t T, int32_t max_em, double tol, float* map_out, double* logpost)
{
    if (!c) return fail(nullptr, SPA_EINVAL, "ctx is NULL");
    if (!map_out || T < 1 || max_em < 1 || !(tol > 0.0)) return fail(c, SPA_EINVAL, "bad arguments");
    if (c->best_T != T || c->rb.T != T || !c->rb.best)
        return fail(c, SPA_EINVAL, "no recorded run of T steps with config.map_path set");
    if (!map_fits(c->n, (int)c->p)) return fail(c, SPA_EINVAL, "n + 5p too large for the MAP solver's shared memory");
    return map_path_impl(c, c->rb.best, c->rb.sched, T, max_em, tol, map_out, logpost);
}

int spa_map_path_given(spa_ctx* c, const double* sched, const float* best, int64_t T, int32_t max_em, double tol,
                       float* map_out, double* logpost)
{
    if (!c) return fail(nullptr, SPA_EINVAL, "ctx is NULL");
    if (!sched || !best || !map_out || T < 1 || T > (int64_t)1 << 24 || max_em < 1 || !(tol > 0.0))
        return fail(c, SPA_EINVAL, "bad arguments");
    for (int64_t t = 0; t < T; ++t)
        if (!(sched[t] > 0.0) || !std::isfinite(sched[t])) return fail(c, SPA_EINVAL, "schedule values must be finite and > 0");
    if (!map_fits(c->n, (int)c->p)) return fail(c, SPA_EINVAL, "n + 5p too large for the MAP solver's shared memory");
    const int64_t p = c->p;
    cudaStream_t st = c->stream();
    double* d_sched = nullptr;
    float* d_best = nullptr;
    cudaError_t e = dalloc(&d_sched, (size_t)T);
    if (e == cudaSuccess) e = dalloc(&d_best, (size_t)(T * p));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_sched, sched, sizeof(double) * (size_t)T, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_best, best, sizeof(float) * (size_t)(T * p), cudaMemcpyHostToDevice, st);
    int rc = e == cudaSuccess ? map_path_impl(c, d_best, d_sched, T, max_em, tol, map_out, logpost)
                              : cuda_fail(c, e, "MAP path inputs");
    cudaStreamSynchronize(st);
    dfree(d_sched);
    dfree(d_best);
    return rc;
}

int spa_map_path_rounds(const spa_ctx* c) { return c ? c->map_rounds : -1; }

int spa_loglik(spa_ctx* c, const float* B, int64_t N, double* ll_out)
{
    return loglik_impl(c, B, false, N, ll_out, false, nullptr);
}

int spa_loglik_device(spa_ctx* c, const float* B, int64_t N, double* ll, void* stream)
{
    return loglik_impl(c, B, true, N, ll, true, static_cast<cudaStream_t>(stream));
}

static int grad_impl(spa_ctx* c, const float* B, bool dev, int64_t N, double cs, double* ll, float* grad,
                     cudaStream_t st_user)
{
    if (!c) return fail(nullptr, SPA_EINVAL, "ctx is NULL");
    if (!B || !grad || N < 1 || N > (int64_t)1 << 22) return fail(c, SPA_EINVAL, "bad arguments");
    if (!(cs >= 0.0) || !std::isfinite(cs)) return fail(c, SPA_EINVAL, "c must be >= 0");
    int rc = ensure_workspace(c, N);
    if (rc != SPA_OK) return rc;
    Workspace& w = c->ws;
    const int64_t p = c->p, n = c->n;
    if (c->cfg.precision == SPA_PREC_SPLIT_BF16) {
        rc = ensure_adjoint_buffers(c);
        if (rc != SPA_OK) return rc;
        if (!w.grad) {
            cudaError_t e = dalloc(&w.grad, (size_t)(N * p));
            if (e != cudaSuccess) return cuda_fail(c, e, "gradient buffer");
        }
        cudaStream_t st = st_user ? st_user : c->stream();
        if (st_user) CK(cudaStreamSynchronize(c->stream()), "sync context stream");
        CK(cudaMemcpyAsync(w.beta, B, sizeof(float) * (size_t)(N * p),
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st),
           "copy B");
        Enq q;
        q.c = c;
        q.st = st;
        const MoveArgs a = move_args(c, nullptr);
        q.ck(launch_move_rw(a, false, N, (int)p, c->pr, c->unit_k, 0, 0u, 0u, nullptr, 0, c->d_err, st));
        enq_grad_tc(q, dev ? grad : w.grad, w.beta, cs, N);
        q.ck(launch_finish_loglik(a.mh, N, nullptr, (dev && ll) ? ll : w.ll, c->d_err, st));
        if (q.e != cudaSuccess) return cuda_fail(c, q.e, "gradient (tensor cores)");
        if (!dev) {
            CK(cudaMemcpyAsync(grad, w.grad, sizeof(float) * (size_t)(N * p), cudaMemcpyDeviceToHost, st), "copy grad");
            if (ll) CK(cudaMemcpyAsync(ll, w.ll, sizeof(double) * (size_t)N, cudaMemcpyDeviceToHost, st), "copy ll");
        }
        CK(cudaStreamSynchronize(st), "sync");
        return read_error_word(c);
    }
    if (!w.eta) {
        const int64_t tiles = (n + SIMT_TILE_N - 1) / SIMT_TILE_N;
        cudaError_t e = dalloc(&w.eta, (size_t)(N * n + tiles * N));
        if (e == cudaSuccess) e = dalloc(&w.grad, (size_t)(N * p));
        if (e != cudaSuccess) return cuda_fail(c, e, "gradient scratch");
    }
    cudaStream_t st = st_user ? st_user : c->stream();
    if (st_user) CK(cudaStreamSynchronize(c->stream()), "sync context stream");
    CK(cudaMemcpyAsync(w.beta, B, sizeof(float) * (size_t)(N * p), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st),
       "copy B");
    CK(launch_grad_simt(w.beta, c->Xf, c->y, N, n, (int)p, w.eta, dev ? grad : w.grad, dev ? ll : (ll ? w.ll : nullptr),
                        c->pr, cs, st),
       "gradient");
    if (!dev) {
        CK(cudaMemcpyAsync(grad, w.grad, sizeof(float) * (size_t)(N * p), cudaMemcpyDeviceToHost, st), "copy grad");
        if (ll) CK(cudaMemcpyAsync(ll, w.ll, sizeof(double) * (size_t)N, cudaMemcpyDeviceToHost, st), "copy ll");
    }
    CK(cudaStreamSynchronize(st), "sync");
    return read_error_word(c);
}

int spa_grad(spa_ctx* c, const float* B, int64_t N, double cs, double* ll_out, float* grad_out)
{
    return grad_impl(c, B, false, N, cs, ll_out, grad_out, nullptr);
}

int spa_grad_device(spa_ctx* c, const float* B, int64_t N, double cs, double* ll, float* grad, void* stream)
{
    return grad_impl(c, B, true, N, cs, ll, grad, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

// ------------------------------------------------------- context-free entry points
namespace {

struct Scratch {
    std::vector<void*> ptrs;
    ~Scratch()
    {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    T* get(size_t count)
    {
        void* p = nullptr;
        if (cudaMalloc(&p, (count ? count : 1) * sizeof(T)) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
};

int finish_free(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamPerThread);
    if (e != cudaSuccess) return fail(nullptr, e == cudaErrorMemoryAllocation ? SPA_ENOMEM : SPA_ECUDA,
                                      std::string(what) + ": " + cudaGetErrorString(e));
    return SPA_OK;
}

}  // namespace

extern "C" {

int spa_resample_systematic(const double* W, int64_t N, double u, int32_t* idx)
{
    if (!W || !idx || N < 1 || N > (int64_t)1 << 24 || !(u >= 0.0 && u < 1.0))
        return fail(nullptr, SPA_EINVAL, "bad arguments");
    if (check_device(nullptr) != SPA_OK) return SPA_EUNSUPPORTED;
    Scratch s;
    double* dW = s.get<double>(N);
    double* dC = s.get<double>(N + (N + 255) / 256 + 1);
    int32_t* dI = s.get<int32_t>(N);
    if (!dW || !dC || !dI) return fail(nullptr, SPA_ENOMEM, "device allocation");
    cudaStream_t st = cudaStreamPerThread;
    cudaError_t e = cudaMemcpyAsync(dW, W, sizeof(double) * (size_t)N, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_resample_index(dW, N, dC, dI, nullptr, 0, nullptr, u, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(idx, dI, sizeof(int32_t) * (size_t)N, cudaMemcpyDeviceToHost, st);
    return finish_free(e, "resample");
}

int spa_prior_logpdf(double nu, double cs, const float* beta, int64_t k, double* out)
{
    if (!beta || !out || k < 0 || !(nu > 0.0) || !(cs > 0.0) || !std::isfinite(cs))
        return fail(nullptr, SPA_EINVAL, "bad arguments");
    if (k == 0) return SPA_OK;
    if (check_device(nullptr) != SPA_OK) return SPA_EUNSUPPORTED;
    PriorArgs pr{std::isinf(nu) ? 1.0f : (float)nu, std::isinf(nu) ? 1 : 0};
    Scratch s;
    float* dB = s.get<float>(k);
    double* dO = s.get<double>(k);
    if (!dB || !dO) return fail(nullptr, SPA_ENOMEM, "device allocation");
    cudaStream_t st = cudaStreamPerThread;
    cudaError_t e = cudaMemcpyAsync(dB, beta, sizeof(float) * (size_t)k, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_prior_logpdf(pr, cs, dB, k, dO, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dO, sizeof(double) * (size_t)k, cudaMemcpyDeviceToHost, st);
    return finish_free(e, "prior logpdf");
}

int spa_incr_weight(double nu, double c_prev, double c_new, const float* B, int64_t N, int64_t p, double* out)
{
    if (!B || !out || N < 1 || p < 1 || !(nu > 0.0) || !(c_prev > 0.0) || !(c_new > 0.0) || !std::isfinite(c_prev) ||
        !std::isfinite(c_new))
        return fail(nullptr, SPA_EINVAL, "bad arguments");
    if (check_device(nullptr) != SPA_OK) return SPA_EUNSUPPORTED;
    PriorArgs pr{std::isinf(nu) ? 1.0f : (float)nu, std::isinf(nu) ? 1 : 0};
    Scratch s;
    float* dB = s.get<float>(N * p);
    double* dW = s.get<double>(N);
    float2* dL = s.get<float2>(N);
    double* dS = s.get<double>(2);
    uint32_t* dE = s.get<uint32_t>(1);
    float4* dK = s.get<float4>(2);
    ReweightK* dR = s.get<ReweightK>(2);
    if (!dB || !dW || !dL || !dS || !dE || !dK || !dR) return fail(nullptr, SPA_ENOMEM, "device allocation");
    cudaStream_t st = cudaStreamPerThread;
    const double sched[2] = {c_prev, c_new};
    cudaError_t e = cudaMemcpyAsync(dB, B, sizeof(float) * (size_t)(N * p), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dS, sched, sizeof(sched), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dW, 0, sizeof(double) * (size_t)N, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dE, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) e = launch_step_constants(pr, dS, 2, (int)p, dK, dR, st);
    if (e == cudaSuccess) e = launch_reweight(dB, dW, dL, N, (int)p, pr, dR, 1, dE, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dW, sizeof(double) * (size_t)N, cudaMemcpyDeviceToHost, st);
    return finish_free(e, "incremental weight");
}

int spa_marginal(const double* log_z_inc, const double* mean, const double* conc, int64_t T, int64_t p, int32_t D,
                 double* post_c, double* mean_out, double* conc_out)
{
    if (!log_z_inc || !mean || !post_c || !mean_out || T < 1 || p < 1 || D < 0 || D > SPA_MAX_DELTAS ||
        (D > 0 && (!conc || !conc_out)))
        return fail(nullptr, SPA_EINVAL, "bad arguments");
    if (check_device(nullptr) != SPA_OK) return SPA_EUNSUPPORTED;
    Scratch s;
    double* dZ = s.get<double>(T);
    double* dM = s.get<double>(T * p);
    double* dC = s.get<double>(T * p * (D > 0 ? D : 1));
    double* dP = s.get<double>(T);
    double* dMo = s.get<double>(p);
    double* dCo = s.get<double>(p * (D > 0 ? D : 1));
    if (!dZ || !dM || !dC || !dP || !dMo || !dCo) return fail(nullptr, SPA_ENOMEM, "device allocation");
    cudaStream_t st = cudaStreamPerThread;
    cudaError_t e = cudaMemcpyAsync(dZ, log_z_inc, sizeof(double) * (size_t)T, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dM, mean, sizeof(double) * (size_t)(T * p), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && D > 0)
        e = cudaMemcpyAsync(dC, conc, sizeof(double) * (size_t)(T * p * D), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_marginal(dZ, dM, dC, T, p, D, dP, dMo, dCo, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(post_c, dP, sizeof(double) * (size_t)T, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mean_out, dMo, sizeof(double) * (size_t)p, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && D > 0)
        e = cudaMemcpyAsync(conc_out, dCo, sizeof(double) * (size_t)(p * D), cudaMemcpyDeviceToHost, st);
    return finish_free(e, "marginal");
}

int spa_marginal_device(const double* log_z_inc, const double* mean, const double* conc, int64_t T, int64_t p,
                        int32_t D, double* post_c, double* mean_out, double* conc_out, void* stream)
{
    if (!log_z_inc || !mean || !post_c || !mean_out || T < 1 || p < 1 || D < 0 || D > SPA_MAX_DELTAS ||
        (D > 0 && (!conc || !conc_out)))
        return fail(nullptr, SPA_EINVAL, "bad arguments");
    if (check_device(nullptr) != SPA_OK) return SPA_EUNSUPPORTED;
    const cudaError_t e = launch_marginal(log_z_inc, mean, conc, T, p, D, post_c, mean_out, conc_out,
                                          static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(nullptr, SPA_ECUDA, std::string("marginal: ") + cudaGetErrorString(e));
    return SPA_OK;
}

int spa_lse_ess(const double* logw, int64_t N, double* lse, double* ess)
{
    if (!logw || N < 1) return fail(nullptr, SPA_EINVAL, "bad arguments");
    if (check_device(nullptr) != SPA_OK) return SPA_EUNSUPPORTED;
    Scratch s;
    double* dL = s.get<double>(N);
    double* dW = s.get<double>(N);
    float* dWf = s.get<float>(N);
    uint32_t* dFix = s.get<uint32_t>(N);
    double* dS = s.get<double>(LSE_SCRATCH);
    unsigned int* dC = s.get<unsigned int>(1);
    double* dOut = s.get<double>(2);
    uint8_t* dR = s.get<uint8_t>(1);
    int* dF = s.get<int>(1);
    uint32_t* dE = s.get<uint32_t>(1);
    if (!dL || !dW || !dWf || !dFix || !dS || !dC || !dOut || !dR || !dF || !dE)
        return fail(nullptr, SPA_ENOMEM, "device allocation");
    cudaStream_t st = cudaStreamPerThread;
    const WeightArrays wa{dL, dW, dWf, dFix};
    cudaError_t e = cudaMemcpyAsync(dL, logw, sizeof(double) * (size_t)N, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dE, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dC, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) e = launch_lse_ess(wa, N, dS, dC, 0, 0, 0.0, dOut + 1, dOut, dR, dF, dE, st);
    double h[2] = {0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, dOut, sizeof(h), cudaMemcpyDeviceToHost, st);
    int rc = finish_free(e, "lse/ess");
    if (rc != SPA_OK) return rc;
    if (lse) *lse = h[0];
    if (ess) *ess = h[1];
    return SPA_OK;
}

int spa_summaries(const float* B, const double* W, int64_t N, int64_t p, const double* q, int32_t nq,
                  const double* deltas, int32_t nd, double* mean, double* quant, double* conc)
{
    if (!B || !W || N < 1 || p < 1 || nq < 0 || nq > 8 || nd < 0 || nd > 8 || (nq && !q) || (nd && !deltas))
        return fail(nullptr, SPA_EINVAL, "bad arguments");
    if (check_device(nullptr) != SPA_OK) return SPA_EUNSUPPORTED;
    SummaryArgs sa;
    sa.nq = nq;
    sa.nd = nd;
    for (int k = 0; k < 8; ++k) {
        sa.q[k] = k < nq ? q[k] : 0.5;
        sa.delta[k] = k < nd ? deltas[k] : 1.0;
    }
    Scratch s;
    float* dB = s.get<float>(N * p);
    double* dW = s.get<double>(N);
    float* dWf = s.get<float>(N);
    uint32_t* dFix = s.get<uint32_t>(N);
    double* dM = s.get<double>(p);
    double* dQ = s.get<double>(p * (nq ? nq : 1));
    double* dC = s.get<double>(p * (nd ? nd : 1));
    uint32_t* dK = s.get<uint32_t>(N * p);
    if (!dB || !dW || !dWf || !dFix || !dM || !dQ || !dC || !dK) return fail(nullptr, SPA_ENOMEM, "device allocation");
    cudaStream_t st = cudaStreamPerThread;
    cudaError_t e = cudaMemcpyAsync(dB, B, sizeof(float) * (size_t)(N * p), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dW, W, sizeof(double) * (size_t)N, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_weight_forms(dW, N, dWf, dFix, st);
    if (e == cudaSuccess) e = launch_summaries(dB, dWf, dFix, N, (int)p, sa, 0, dM, nq ? dQ : nullptr, dC, dK, st);
    if (e == cudaSuccess && mean) e = cudaMemcpyAsync(mean, dM, sizeof(double) * (size_t)p, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && quant && nq)
        e = cudaMemcpyAsync(quant, dQ, sizeof(double) * (size_t)(p * nq), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && conc && nd)
        e = cudaMemcpyAsync(conc, dC, sizeof(double) * (size_t)(p * nd), cudaMemcpyDeviceToHost, st);
    return finish_free(e, "summaries");
}

int spa_philox4x32_10(const uint32_t* ctr, const uint32_t* key, int64_t count, uint32_t* out)
{
    if (!ctr || !key || !out || count < 0) return fail(nullptr, SPA_EINVAL, "bad arguments");
    if (count == 0) return SPA_OK;
    if (check_device(nullptr) != SPA_OK) return SPA_EUNSUPPORTED;
    Scratch s;
    uint32_t* dC = s.get<uint32_t>(4 * count);
    uint32_t* dO = s.get<uint32_t>(4 * count);
    if (!dC || !dO) return fail(nullptr, SPA_ENOMEM, "device allocation");
    cudaStream_t st = cudaStreamPerThread;
    cudaError_t e = cudaMemcpyAsync(dC, ctr, sizeof(uint32_t) * 4 * (size_t)count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_philox(dC, make_uint2(key[0], key[1]), count, dO, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dO, sizeof(uint32_t) * 4 * (size_t)count, cudaMemcpyDeviceToHost, st);
    return finish_free(e, "philox");
}

int spa_normals(uint64_t seed, uint32_t particle, uint32_t t, uint32_t m, int64_t p, float* out)
{
    if (!out || p < 1) return fail(nullptr, SPA_EINVAL, "bad arguments");
    if (check_device(nullptr) != SPA_OK) return SPA_EUNSUPPORTED;
    Scratch s;
    float* dO = s.get<float>(p);
    if (!dO) return fail(nullptr, SPA_ENOMEM, "device allocation");
    cudaStream_t st = cudaStreamPerThread;
    cudaError_t e = launch_normals(seed, particle, t, m, p, dO, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dO, sizeof(float) * (size_t)p, cudaMemcpyDeviceToHost, st);
    return finish_free(e, "normals");
}

int spa_prior_sample(uint64_t seed, double nu, double cs, int64_t N, int64_t p, float* out)
{
    if (!out || N < 1 || p < 1 || !(nu > 0.0) || !(cs > 0.0)) return fail(nullptr, SPA_EINVAL, "bad arguments");
    if (check_device(nullptr) != SPA_OK) return SPA_EUNSUPPORTED;
    PriorArgs pr{std::isinf(nu) ? 1.0f : (float)nu, std::isinf(nu) ? 1 : 0};
    Scratch s;
    float* dO = s.get<float>(N * p);
    if (!dO) return fail(nullptr, SPA_ENOMEM, "device allocation");
    cudaStream_t st = cudaStreamPerThread;
    cudaError_t e = launch_prior_sample(seed, pr, cs, N, p, dO, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dO, sizeof(float) * (size_t)(N * p), cudaMemcpyDeviceToHost, st);
    return finish_free(e, "prior sample");
}

}  // extern "C"
