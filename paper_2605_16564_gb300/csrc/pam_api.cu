// pam_api.cu -- host side of libpam: argument validation, sizes, workspace
// carve-up and the order of the launches of each C-ABI entry point.
#include <cmath>
#include <cstring>
#include <atomic>
#include <mutex>
#include <vector>

#include <cfloat>

#include "pam_internal.cuh"

namespace pam {

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static int64_t prod3(const int v[3]) { return (int64_t)v[0] * v[1] * v[2]; }

// Validates a problem/parameter pair and fills the kernel-side view.
// `par` may be NULL (calls that need only the geometry).
bool make_geo(const pam_problem *prob, const pam_params *par, Geo *g, Par *p, pam_status *st) {
    *st = PAM_ERR_INVALID_ARG;
    if (!prob) return false;
    *g = Geo{};  // zeros, and every subdomain in one group (stride 1)
    if (prob->dim < 1 || prob->dim > 3) return false;
    g->dim = prob->dim;
    int64_t S = 1, nmax = 1;
    for (int a = 0; a < 3; ++a) {
        bool used = a < prob->dim;
        g->n[a] = used ? prob->n_cells[a] : 1;
        g->p[a] = used ? prob->n_sub[a] : 1;
        g->g[a] = used ? prob->g_init[a] : 1;
        if (g->n[a] < 1 || g->n[a] > (1 << 24)) return false;
        if (g->p[a] < 1 || g->p[a] > g->n[a]) return false;
        if (g->g[a] < 1) return false;
        S *= g->p[a];
        if (g->n[a] > nmax) nmax = g->n[a];
    }
    if (prob->overlap < 0) return false;
    if (S > 65535) return false;
    if (prod3(g->n) > ((int64_t)1 << 40)) return false;
    g->overlap = prob->overlap;
    g->S = (int)S;
    g->sub_lo = 0;
    g->sub_hi = (int)S;
    g->nmax = (int)nmax;
    g->h = 1.0 / (double)nmax;
    g->vol = 1.0;
    for (int a = 0; a < g->dim; ++a) g->vol *= g->h;
    // largest patch: the widest core along each axis grown by the overlap
    int64_t nm = 1;
    for (int a = 0; a < 3; ++a) {
        int widest = 0;
        for (int j = 0; j < g->p[a]; ++j) {
            int64_t lo = ((int64_t)j * g->n[a]) / g->p[a], hi = ((int64_t)(j + 1) * g->n[a]) / g->p[a];
            int64_t plo = lo - (a < g->dim ? g->overlap : 0), phi = hi + (a < g->dim ? g->overlap : 0);
            if (plo < 0) plo = 0;
            if (phi > g->n[a]) phi = g->n[a];
            if (phi - plo > widest) widest = (int)(phi - plo);
        }
        nm *= widest;
    }
    if (nm > (1 << 20)) { *st = PAM_ERR_UNSUPPORTED; return false; }
    g->n_max = (int)align_up((size_t)nm, 32);
    g->m0 = (int)prod3(g->g);
    if (g->m0 > PAM_MAX_M) { *st = PAM_ERR_UNSUPPORTED; return false; }
    g->m_cap = (int)align_up((size_t)g->m0, 64);
    if (par) {
        if (!(par->lambda1_hat >= 0.0) || !(par->lambda2_hat > 0.0)) return false;
        if (!std::isfinite(par->lambda1_hat) || !std::isfinite(par->lambda2_hat)) return false;
        if (!(par->eta > 0.0 && par->eta < 1.0)) return false;
        if (std::isnan(par->eps_tol_rel)) return false;
        if (par->k_top < 0 || par->m_max < 0 || par->levels < 0 || par->max_iters < 0) return false;
        if (par->warm_start != 0 && par->warm_start != 1) return false;
        if (par->quad != 0 && par->quad != 1) return false;
        if (par->deferred_status != 0 && par->deferred_status != 1) return false;
        if (par->precision != PAM_PREC_FP64 && par->precision != PAM_PREC_MIXED) return false;
        if (par->sub_begin < 0 || par->sub_end < par->sub_begin || par->sub_end > g->S) return false;
        if (par->sub_end > 0) {
            g->sub_lo = par->sub_begin;
            g->sub_hi = par->sub_end;
        }
        int64_t add = (int64_t)par->levels * (g->dim + 1) * par->k_top;
        if (add > par->m_max) add = par->m_max;
        int64_t cap = (int64_t)g->m0 + add;
        cap = (int64_t)align_up((size_t)cap, 64);
        if (cap > PAM_MAX_M) { *st = PAM_ERR_UNSUPPORTED; return false; }
        // the tensor-core Gram keeps a 128 x M strip in TMEM (512 columns)
        if (par->precision == PAM_PREC_MIXED && cap > kMixedMaxM) { *st = PAM_ERR_UNSUPPORTED; return false; }
        // marking sorts a patch's keys in shared memory: 2^ceil(log2 N) x 8 bytes
        if (par->levels > 0) {
            int64_t P = 1;
            while (P < g->n_max) P <<= 1;
            if (P * 8 > 227 * 1024) { *st = PAM_ERR_UNSUPPORTED; return false; }
        }
        g->m_cap = (int)cap;
        g->prec = par->precision;
        if (p) {
            p->lam1_hat = par->lambda1_hat;
            p->lam2_hat = par->lambda2_hat;
            p->eps_tol_rel = par->eps_tol_rel;
            p->eta = par->eta;
            p->k_top = par->k_top;
            p->m_max = par->m_max;
            p->levels = par->levels;
            p->max_iters = par->max_iters > 0 ? par->max_iters : 200;
            p->quad = par->quad;
            p->cv_folds = 0;
            p->cv_fold = 0;
        }
    }
    *st = PAM_OK;
    return true;
}

// Region sizes. Small regions come first so that calls which use only them
// (errors) agree with the fit calls on where they live.
static size_t carve(const Geo &g, char *base, Ws *w) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off = align_up(off + bytes, 256);
        return p;
    };
    const size_t S = (size_t)g.S, nm = (size_t)g.n_max, mc = (size_t)g.m_cap;
    w->status = (int32_t *)take(8 * sizeof(int32_t));
    w->kmax_bits = (unsigned long long *)take(S * sizeof(unsigned long long));
    w->err_part = (double *)take((S > (size_t)kErrBlocks ? S : (size_t)kErrBlocks) * 8 * sizeof(double));
    w->y = (double *)take(S * nm * sizeof(double));
    w->kv = (double *)take(S * nm * sizeof(double));
    w->inv_s = (double *)take(S * nm * sizeof(double));
    w->R = (double *)take(S * nm * sizeof(double));
    w->rowmax = (float *)take(S * nm * sizeof(float));
    w->rowinv = (float *)take(S * nm * sizeof(float));
    w->b = (double *)take(S * mc * sizeof(double));
    w->wsum = (float *)take(S * mc * sizeof(float));
    w->cost = (uint32_t *)take(S * sizeof(uint32_t));
    w->order = (int32_t *)take(S * sizeof(int32_t));
    // large regions: the fp64 form needs E, G and fp64 factors; the mixed
    // form only its fp32 Gram and fp32 factors
    const bool f64 = g.prec == PAM_PREC_FP64;
    w->L = (double *)take(S * (mc * (mc + 1) / 2) * (f64 ? sizeof(double) : sizeof(float)));
    w->Lf = (float *)w->L;
    w->G = (double *)take(S * mc * mc * (f64 ? sizeof(double) : sizeof(float)));
    w->Gf = (float *)w->G;
    w->E = f64 ? (double *)take(S * mc * nm * sizeof(double)) : nullptr;
    w->cxv = g.cells ? (double4_32a *)take(S * nm * sizeof(double4_32a)) : nullptr;
    // the mixed form's binary64 fallback: a list and min(S, kFbSlots) slots
    w->bytes_no_fb = off;
    const size_t F = f64 ? 0 : (S < (size_t)kFbSlots ? S : (size_t)kFbSlots);
    w->fb_slots = (int)F;
    // (4 + F: room for two lists when the subdomains run in two groups)
    w->fb = F ? (int32_t *)take((4 + F) * sizeof(int32_t)) : nullptr;
    w->fbE = F ? (double *)take(F * mc * nm * sizeof(double)) : nullptr;
    w->fbG = F ? (double *)take(F * mc * mc * sizeof(double)) : nullptr;
    w->fbL = F ? (double *)take(F * (mc * (mc + 1) / 2) * sizeof(double)) : nullptr;
    w->bytes = off;
    return off;
}

// ---------------------------------------------------------------- timing ---
// Event pairs recorded on the launching stream; read back (with one
// synchronisation) by pam_timing_read.
namespace {
struct Pair {
    int phase;
    cudaEvent_t a, b;
};
bool g_timing = false;
std::atomic<long long> g_launches{0};
std::vector<Pair> g_pairs;
std::mutex g_mu;
}  // namespace

void count_launches(int n) { g_launches += n; }

PhaseScope::PhaseScope(int phase, cudaStream_t st)
    : phase_(phase), st_(st), stop_(nullptr), on_(g_timing), capturing_(false) {
    if (!on_) return;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    // inside a stream capture the pair becomes event-record nodes of the
    // graph, re-recorded by every replay (read them after each replay)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    capturing_ = cs == cudaStreamCaptureStatusActive;
    if (capturing_) cudaEventRecordWithFlags(a, st, cudaEventRecordExternal);
    else cudaEventRecord(a, st);
    stop_ = b;
    std::lock_guard<std::mutex> lk(g_mu);
    g_pairs.push_back({phase, a, b});
}

PhaseScope::~PhaseScope() {
    if (!on_) return;
    if (capturing_) cudaEventRecordWithFlags(stop_, st_, cudaEventRecordExternal);
    else cudaEventRecord(stop_, st_);
}

Ws carve_workspace(const Geo &g, void *base) {
    Ws w;
    carve(g, (char *)base, &w);
    return w;
}

}  // namespace pam

namespace pam {
static pam_tuning g_tuning = {0, 0, 0, 0, 0, {0, 0, 0}};  // factor_kb, gram_stages, eval_block, persistent, groups
const pam_tuning &tuning() { return g_tuning; }

// Median of three timed runs of `body` (after one untimed run) on `st`, ms.
template <class F>
static pam_status time_median(cudaStream_t st, F body, double *ms) {
    cudaEvent_t a, b;
    PAM_CUDA_TRY(cudaEventCreate(&a));
    PAM_CUDA_TRY(cudaEventCreate(&b));
    body();
    float t[3];
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(a, st);
        body();
        cudaEventRecord(b, st);
        if (cudaEventSynchronize(b) != cudaSuccess) {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            return PAM_ERR_CUDA;
        }
        cudaEventElapsedTime(&t[r], a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    const float lo = fminf(t[0], fminf(t[1], t[2])), hi = fmaxf(t[0], fmaxf(t[1], t[2]));
    *ms = (double)(t[0] + t[1] + t[2] - lo - hi);
    PAM_CUDA_TRY(cudaGetLastError());
    return PAM_OK;
}

}  // namespace pam

using namespace pam;

extern "C" {

const char *pam_version(void) { return "libpam 0.1 (sm_103a)"; }

int pam_struct_sizes(size_t *out, int n) {
    const size_t sz[6] = {sizeof(pam_problem), sizeof(pam_params), sizeof(pam_plan),
                          sizeof(pam_model),   sizeof(pam_cells),  sizeof(pam_tuning)};
    for (int i = 0; out && i < n && i < 6; ++i) out[i] = sz[i];
    return 6;
}

void pam_timing_enable(int on) { g_timing = on != 0; }

long long pam_kernel_launches(void) { return g_launches.load(); }

void pam_timing_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &p : g_pairs) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    g_pairs.clear();
}

pam_status pam_timing_read(int phase, double *h_total_ms, int *h_count) {
    if (!h_total_ms || !h_count || phase < 0 || phase >= PAM_PHASE_COUNT) return PAM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    double tot = 0.0;
    int cnt = 0;
    for (auto &p : g_pairs) {
        if (p.phase != phase) continue;
        if (cudaEventSynchronize(p.b) != cudaSuccess) return PAM_ERR_CUDA;
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) return PAM_ERR_CUDA;
        tot += ms;
        ++cnt;
    }
    *h_total_ms = tot;
    *h_count = cnt;
    return PAM_OK;
}

const char *pam_status_string(pam_status s) {
    switch (s) {
        case PAM_OK: return "ok";
        case PAM_ERR_INVALID_ARG: return "invalid argument";
        case PAM_ERR_NONPOSITIVE_K: return "cell value <= 0, NaN or Inf";
        case PAM_ERR_CUDA: return "CUDA runtime error";
        case PAM_ERR_WORKSPACE: return "workspace too small";
        case PAM_ERR_NOT_CONVERGED: return "a subdomain solve was not certified";
        case PAM_ERR_UNSUPPORTED: return "unsupported size";
        case PAM_ERR_TIMEOUT: return "a device wait ran out of time";
    }
    return "unknown status";
}

pam_status pam_plan_create(const pam_problem *prob, const pam_params *par, pam_plan *out) {
    if (!prob || !par || !out) return PAM_ERR_INVALID_ARG;
    Geo g;
    Par p;
    pam_status st;
    if (!make_geo(prob, par, &g, &p, &st)) return st;
    Ws w;
    out->n_subdomains = g.S;
    out->max_patch_cells = g.n_max;
    out->m0 = g.m0;
    out->m_cap = g.m_cap;
    out->n_grid_cells = prod3(g.n);
    out->workspace_bytes = carve(g, nullptr, &w);
    return PAM_OK;
}

pam_status pam_partition(const pam_problem *prob, int32_t *h_boxes) {
    if (!prob || !h_boxes) return PAM_ERR_INVALID_ARG;
    Geo g;
    pam_status st;
    if (!make_geo(prob, nullptr, &g, nullptr, &st)) return st;
    for (int s = 0; s < g.S; ++s) {
        int j[3] = {s % g.p[0], (s / g.p[0]) % g.p[1], s / (g.p[0] * g.p[1])};
        for (int a = 0; a < 3; ++a) {
            int lo = (int)(((int64_t)j[a] * g.n[a]) / g.p[a]);
            int hi = (int)(((int64_t)(j[a] + 1) * g.n[a]) / g.p[a]);
            int ov = a < g.dim ? g.overlap : 0;
            h_boxes[s * 12 + a] = lo;
            h_boxes[s * 12 + 3 + a] = hi;
            h_boxes[s * 12 + 6 + a] = lo - ov < 0 ? 0 : lo - ov;
            h_boxes[s * 12 + 9 + a] = hi + ov > g.n[a] ? g.n[a] : hi + ov;
        }
    }
    return PAM_OK;
}

static bool model_ok(const pam_model *m) {
    return m && m->boxes && m->centres && m->beta && m->info;
}

static pam_status check_plan(const Geo &g, const pam_plan *plan) {
    if (!plan) return PAM_ERR_INVALID_ARG;
    if (plan->n_subdomains != g.S || plan->m_cap < g.m_cap || plan->max_patch_cells != g.n_max ||
        plan->m_cap > PAM_MAX_M || plan->m_cap % 64 != 0)
        return PAM_ERR_INVALID_ARG;
    return PAM_OK;
}

// Reads the device status words after the enqueued work (one sync).
static pam_status read_status(const Ws &w, cudaStream_t st, int32_t host[8]) {
    PAM_CUDA_TRY(cudaMemcpyAsync(host, w.status, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PAM_CUDA_TRY(cudaStreamSynchronize(st));
    return PAM_OK;
}

// Step 2 launches shared by the grid and the element-list entry points.
// Subdomain groups of the levels (the initial lattices' solve in
// pam_fit_subdomains, the refinement levels in pam_refine). Each level is
// (marking ->) statistics -> Gram -> solve over every subdomain, and the solve's last
// subdomains leave most of the SMs idle while they finish (its costs vary
// severalfold from subdomain to subdomain and are not known before it runs).
// Split into two groups (even and odd subdomain indices, so that both hold
// the same mix of the field), each group runs its levels in order on its own
// stream: one group's solve tail overlaps the other group's marking, Gram
// and solve. The subdomains are independent (section 2), so the results are
// the same bits as one pipeline's. Each group has its own part of the solve
// order and its own half of the binary64 fallback's slots.
constexpr int kGroupMinS = 1024;  // below this the solve has few waves to balance

static int level_groups(const Geo &g, const pam_params *par, const Ws &w, bool timing = g_timing) {
    if (par->precision != PAM_PREC_MIXED || w.fb_slots < 2) return 1;
    if (timing) return 1;  // the phase profiler times one pipeline, phase by phase
    if (g_tuning.level_groups == 1 || g_tuning.level_groups == 2) return g_tuning.level_groups;
    return g.S >= kGroupMinS ? 2 : 1;
}

// Group q of ng: its subdomains gb + i gs (i < gn), the offset of its solve
// order in the order region, of its fallback list in the list region (two
// counters, then the slots' subdomains), its slots and the first of them.
struct GroupLayout {
    int gb, gs, gn, order_off, list_off, slots, slot0;
};

static GroupLayout group_layout(int S, int F, int q, int ng) {
    if (ng == 1) return {0, 1, S, 0, 0, F, 0};
    const int f0 = (F + 1) / 2;  // the even group is the larger one when S is odd
    if (q == 0) return {0, 2, (S + 1) / 2, 0, 0, f0, 0};
    return {1, 2, S / 2, (S + 1) / 2, 2 + f0, F - f0, f0};
}

static Geo group_geo(const Geo &g, int q) {
    const GroupLayout l = group_layout(g.S, 0, q, 2);
    Geo v = g;
    v.gb = l.gb;
    v.gs = l.gs;
    v.gn = l.gn;
    return v;
}

static Ws group_ws(const Geo &g, const Ws &w, int q) {
    const GroupLayout l = group_layout(g.S, w.fb_slots, q, 2);
    const size_t mc = (size_t)g.m_cap, nm = (size_t)g.n_max;
    Ws v = w;
    v.order = w.order + l.order_off;
    v.fb = w.fb + l.list_off;
    v.fb_slots = l.slots;
    v.fbE = w.fbE + (size_t)l.slot0 * mc * nm;
    v.fbG = w.fbG + (size_t)l.slot0 * mc * mc;
    v.fbL = w.fbL + (size_t)l.slot0 * (mc * (mc + 1) / 2);
    return v;
}

// The second group's stream and the fork / join events, one set per host
// thread and device (created on first use, kept for the process).
struct GroupStreams {
    cudaStream_t st = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

static pam_status group_streams(GroupStreams **out) {
    thread_local std::vector<GroupStreams> per_dev;
    int dev = 0;
    PAM_CUDA_TRY(cudaGetDevice(&dev));
    if ((int)per_dev.size() <= dev) per_dev.resize(dev + 1);
    GroupStreams &gs = per_dev[dev];
    if (!gs.st) {
        PAM_CUDA_TRY(cudaStreamCreateWithFlags(&gs.st, cudaStreamNonBlocking));
        PAM_CUDA_TRY(cudaEventCreateWithFlags(&gs.fork, cudaEventDisableTiming));
        PAM_CUDA_TRY(cudaEventCreateWithFlags(&gs.join, cudaEventDisableTiming));
    }
    *out = &gs;
    return PAM_OK;
}

static pam_status fit_launches(const Geo &g, const Par &p, const pam_params *par, const double *d_K,
                               pam_model *model, const Ws &w, cudaStream_t s) {
    pam_status st;
    const bool deferred = par->deferred_status != 0;
    PAM_CUDA_TRY(cudaMemsetAsync(w.status, 0, 8 * sizeof(int32_t), s));
    launch_partition(g, model->boxes, s);
    launch_prepare(g, model->boxes, d_K, w, s);
    PAM_CUDA_TRY(cudaGetLastError());
    int32_t hs[8];
    if (!deferred) {
        if ((st = read_status(w, s, hs)) != PAM_OK) return st;
        if (hs[kStBadK]) return PAM_ERR_NONPOSITIVE_K;
    }
    // a warm start still being written on another stream: the solve waits for
    // it (element lists: the dictionary set-up already, which zeroes the
    // coefficients of a patch without elements)
    cudaEvent_t seeded = par->warm_start ? (cudaEvent_t)par->warm_start_event : nullptr;
    if (seeded && g.cells) {
        PAM_CUDA_TRY(cudaStreamWaitEvent(s, seeded, 0));
        seeded = nullptr;
    }
    launch_init_dictionary(g, model->boxes, model->centres, model->beta, model->info, s,
                           par->warm_start != 0);
    if (par->precision == PAM_PREC_MIXED && level_groups(g, par, w) == 2) {
        // the initial lattices' statistics, Gram and solve in the two groups
        GroupStreams *gs = nullptr;
        if ((st = group_streams(&gs)) != PAM_OK) return st;
        PAM_CUDA_TRY(cudaEventRecord(gs->fork, s));
        PAM_CUDA_TRY(cudaStreamWaitEvent(gs->st, gs->fork, 0));
        const cudaStream_t sq[2] = {s, gs->st};
        for (int q = 0; q < 2; ++q)
            launch_solve_level_mixed(group_geo(g, q), p, model->boxes, model->centres, model->beta, model->info,
                                     group_ws(g, w, q), sq[q], seeded, g.m0);
        PAM_CUDA_TRY(cudaEventRecord(gs->join, gs->st));
        PAM_CUDA_TRY(cudaStreamWaitEvent(s, gs->join, 0));
    } else if (par->precision == PAM_PREC_MIXED)
        launch_solve_level_mixed(g, p, model->boxes, model->centres, model->beta, model->info, w, s, seeded,
                                 g.m0);  // every dictionary is the initial lattice
    else
        launch_solve_level_f64(g, p, model->boxes, model->centres, model->beta, model->info, w, s, seeded);
    PAM_CUDA_TRY(cudaGetLastError());
    if (deferred) return PAM_OK;
    if ((st = read_status(w, s, hs)) != PAM_OK) return st;
    if (hs[kStTimeout]) return PAM_ERR_TIMEOUT;
    return hs[kStUncertified] ? PAM_ERR_NOT_CONVERGED : PAM_OK;
}

pam_status pam_fit_subdomains(const pam_problem *prob, const pam_params *par, const pam_plan *plan,
                              const double *d_K, pam_model *model, void *d_workspace,
                              size_t workspace_bytes, void *stream) {
    Geo g;
    Par p;
    pam_status st;
    if (!par || !make_geo(prob, par, &g, &p, &st)) return par ? st : PAM_ERR_INVALID_ARG;
    if ((st = check_plan(g, plan)) != PAM_OK) return st;
    g.m_cap = plan->m_cap;
    if (par->precision == PAM_PREC_MIXED && (g.m_cap > kMixedMaxM || !mixed_solve_fits(g)))
        return PAM_ERR_UNSUPPORTED;
    if (!d_K || !model_ok(model) || !d_workspace) return PAM_ERR_INVALID_ARG;
    Ws w = carve_workspace(g, d_workspace);
    if (workspace_bytes < w.bytes) return PAM_ERR_WORKSPACE;
    return fit_launches(g, p, par, d_K, model, w, (cudaStream_t)stream);
}

pam_status pam_lambda_cv_workspace_size(const pam_plan *plan, size_t *bytes) {
    if (!plan || !bytes || plan->n_subdomains <= 0 || plan->m_cap <= 0) return PAM_ERR_INVALID_ARG;
    Geo g{};
    g.S = plan->n_subdomains;
    g.m_cap = plan->m_cap;
    *bytes = cv_workspace_bytes(g);
    return PAM_OK;
}

pam_status pam_lambda_cv(const pam_problem *prob, const pam_params *par, const pam_plan *plan,
                         const double *d_K, pam_model *model, const double *h_grid, int n_grid,
                         int n_folds, double *d_cv, int32_t *d_choice, void *d_workspace,
                         size_t workspace_bytes, void *d_cv_workspace, size_t cv_workspace_bytes_,
                         void *stream) {
    Geo g;
    Par p;
    pam_status st;
    if (!par || !make_geo(prob, par, &g, &p, &st)) return par ? st : PAM_ERR_INVALID_ARG;
    if ((st = check_plan(g, plan)) != PAM_OK) return st;
    g.m_cap = plan->m_cap;
    if (par->precision == PAM_PREC_MIXED && (g.m_cap > kMixedMaxM || !mixed_solve_fits(g)))
        return PAM_ERR_UNSUPPORTED;
    if (!d_K || !model_ok(model) || !d_workspace || !h_grid || !d_cv || !d_choice || !d_cv_workspace)
        return PAM_ERR_INVALID_ARG;
    if (n_grid < 1 || n_grid > kCvMaxGrid || n_folds < 2 || n_folds > 1024) return PAM_ERR_INVALID_ARG;
    CvGrid grid{};
    grid.n = n_grid;
    for (int q = 0; q < n_grid; ++q) {
        const double l1 = h_grid[2 * q], l2 = h_grid[2 * q + 1];
        if (!(l1 >= 0.0 && l1 <= DBL_MAX) || !(l2 > 0.0 && l2 <= DBL_MAX)) return PAM_ERR_INVALID_ARG;
        grid.lam[q][0] = l1;
        grid.lam[q][1] = l2;
    }
    Ws w = carve_workspace(g, d_workspace);
    if (workspace_bytes < w.bytes || cv_workspace_bytes_ < cv_workspace_bytes(g)) return PAM_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    PAM_CUDA_TRY(cudaMemsetAsync(w.status, 0, 8 * sizeof(int32_t), s));
    launch_prepare(g, model->boxes, d_K, w, s);
    launch_lambda_cv(g, p, par->precision, model->boxes, model->centres, model->beta, model->info, w, grid,
                     n_folds, d_cv, d_choice, d_cv_workspace, s);
    PAM_CUDA_TRY(cudaGetLastError());
    if (par->deferred_status) return PAM_OK;
    int32_t hs[8];
    if ((st = read_status(w, s, hs)) != PAM_OK) return st;
    if (hs[kStBadK]) return PAM_ERR_NONPOSITIVE_K;
    if (hs[kStTimeout]) return PAM_ERR_TIMEOUT;
    return hs[kStUncertified] ? PAM_ERR_NOT_CONVERGED : PAM_OK;
}

pam_status pam_status_read(const pam_plan *plan, void *d_workspace, size_t workspace_bytes, void *stream) {
    // the status words are the workspace's first region, whatever the problem
    if (!plan || !d_workspace || workspace_bytes < 8 * sizeof(int32_t)) return PAM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t hs[8];
    PAM_CUDA_TRY(cudaMemcpyAsync(hs, d_workspace, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PAM_CUDA_TRY(cudaStreamSynchronize(s));
    if (hs[kStBadK]) return PAM_ERR_NONPOSITIVE_K;
    if (hs[kStTimeout]) return PAM_ERR_TIMEOUT;
    return hs[kStUncertified] ? PAM_ERR_NOT_CONVERGED : PAM_OK;
}

// Step 3 launches shared by the grid and the element-list entry points.
static pam_status refine_launches(const Geo &g, const Par &p, const pam_params *par, pam_model *model,
                                  int n_levels, const Ws &w, cudaStream_t s) {
    pam_status st;
    const bool deferred = par->deferred_status != 0;
    // deferred: the status keeps accumulating from pam_fit_subdomains
    if (!deferred) PAM_CUDA_TRY(cudaMemsetAsync(w.status, 0, 8 * sizeof(int32_t), s));
    const int ng = n_levels > 0 ? level_groups(g, par, w) : 1;
    if (ng == 2) {
        GroupStreams *gs = nullptr;
        if ((st = group_streams(&gs)) != PAM_OK) return st;
        PAM_CUDA_TRY(cudaEventRecord(gs->fork, s));
        PAM_CUDA_TRY(cudaStreamWaitEvent(gs->st, gs->fork, 0));
        const Geo gq[2] = {group_geo(g, 0), group_geo(g, 1)};
        const Ws wq[2] = {group_ws(g, w, 0), group_ws(g, w, 1)};
        const cudaStream_t sq[2] = {s, gs->st};
        for (int lv = 0; lv < n_levels; ++lv)
            for (int q = 0; q < 2; ++q) {
                launch_refine_round(gq[q], p, par->precision, model->boxes, model->centres, model->beta,
                                    model->info, wq[q], sq[q]);
                launch_solve_level_mixed(gq[q], p, model->boxes, model->centres, model->beta, model->info,
                                         wq[q], sq[q]);
            }
        PAM_CUDA_TRY(cudaEventRecord(gs->join, gs->st));
        PAM_CUDA_TRY(cudaStreamWaitEvent(s, gs->join, 0));
    } else {
        for (int lv = 0; lv < n_levels; ++lv) {
            launch_refine_round(g, p, par->precision, model->boxes, model->centres, model->beta,
                                model->info, w, s);
            if (par->precision == PAM_PREC_MIXED)
                launch_solve_level_mixed(g, p, model->boxes, model->centres, model->beta, model->info, w, s);
            else
                launch_solve_level_f64(g, p, model->boxes, model->centres, model->beta, model->info, w, s);
        }
    }
    PAM_CUDA_TRY(cudaGetLastError());
    if (deferred) return PAM_OK;
    int32_t hs[8];
    if ((st = read_status(w, s, hs)) != PAM_OK) return st;
    if (hs[kStTimeout]) return PAM_ERR_TIMEOUT;
    return hs[kStUncertified] ? PAM_ERR_NOT_CONVERGED : PAM_OK;
}

pam_status pam_refine(const pam_problem *prob, const pam_params *par,
                      const pam_plan *plan, const double *d_K, pam_model *model, int n_levels,
                      void *d_workspace, size_t workspace_bytes, void *stream) {
    Geo g;
    Par p;
    pam_status st;
    if (!par || !make_geo(prob, par, &g, &p, &st)) return par ? st : PAM_ERR_INVALID_ARG;
    if ((st = check_plan(g, plan)) != PAM_OK) return st;
    g.m_cap = plan->m_cap;
    if (par->precision == PAM_PREC_MIXED && (g.m_cap > kMixedMaxM || !mixed_solve_fits(g)))
        return PAM_ERR_UNSUPPORTED;
    if (!d_K || !model_ok(model) || !d_workspace || n_levels < 0) return PAM_ERR_INVALID_ARG;
    Ws w = carve_workspace(g, d_workspace);
    if (workspace_bytes < w.bytes) return PAM_ERR_WORKSPACE;
    return refine_launches(g, p, par, model, n_levels, w, (cudaStream_t)stream);
}

pam_status pam_gram(const pam_problem *prob, const pam_params *par, const pam_plan *plan,
                    const double *d_K, const pam_model *model, double *d_G, double *d_b,
                    void *d_workspace, size_t workspace_bytes, void *stream) {
    Geo g;
    Par p;
    pam_status st;
    if (!par || !make_geo(prob, par, &g, &p, &st)) return par ? st : PAM_ERR_INVALID_ARG;
    if ((st = check_plan(g, plan)) != PAM_OK) return st;
    g.m_cap = plan->m_cap;
    if (par->precision == PAM_PREC_MIXED && g.m_cap > kMixedMaxM) return PAM_ERR_UNSUPPORTED;
    if (!d_K || !model_ok(model) || !d_G || !d_b || !d_workspace) return PAM_ERR_INVALID_ARG;
    Ws w = carve_workspace(g, d_workspace);
    if (workspace_bytes < w.bytes_no_fb) return PAM_ERR_WORKSPACE;  // no solve: the fallback slots are not used
    cudaStream_t s = (cudaStream_t)stream;
    PAM_CUDA_TRY(cudaMemsetAsync(w.status, 0, 8 * sizeof(int32_t), s));
    launch_prepare(g, model->boxes, d_K, w, s);
    if (par->precision == PAM_PREC_MIXED) {
        launch_stats_gram_tc(g, model->boxes, model->centres, model->info, w, s, 1);
        launch_copy_gram_f32(g, model->info, w, d_G, d_b, s);
    } else {
        launch_assemble_gram_f64(g, model->boxes, model->centres, model->info, w, s, 1);
        launch_copy_gram_f64(g, model->info, w, d_G, d_b, s);
    }
    PAM_CUDA_TRY(cudaGetLastError());
    int32_t hs[8];
    if ((st = read_status(w, s, hs)) != PAM_OK) return st;
    if (hs[kStBadK]) return PAM_ERR_NONPOSITIVE_K;
    if (hs[kStTimeout]) return PAM_ERR_TIMEOUT;
    return PAM_OK;
}

pam_status pam_eval_workspace_size(const pam_plan *plan, int64_t n_pts, size_t *bytes) {
    if (!plan || !bytes || n_pts < 0 || plan->n_subdomains < 1) return PAM_ERR_INVALID_ARG;
    if (n_pts > (int64_t)INT32_MAX) return PAM_ERR_UNSUPPORTED;
    *bytes = eval_workspace_bytes(plan->n_subdomains, n_pts);
    return PAM_OK;
}

// The argument checks of the evaluation calls (model: NULL for the bucketing).
static pam_status eval_args(const pam_problem *prob, const pam_plan *plan, const pam_model *model,
                            bool need_model, const double *d_pts, int64_t n_pts, double *d_out, int precision,
                            void *d_workspace, size_t workspace_bytes, Geo *g) {
    pam_status st;
    if (!make_geo(prob, nullptr, g, nullptr, &st)) return st;
    if (!plan || plan->n_subdomains != g->S || plan->m_cap > PAM_MAX_M || plan->m_cap < 1)
        return PAM_ERR_INVALID_ARG;
    g->m_cap = plan->m_cap;
    g->n_max = plan->max_patch_cells;
    if (n_pts < 0 || (need_model && !model_ok(model))) return PAM_ERR_INVALID_ARG;
    if (precision != PAM_PREC_FP64 && precision != PAM_PREC_MIXED) return PAM_ERR_INVALID_ARG;
    if (n_pts > (int64_t)INT32_MAX) return PAM_ERR_UNSUPPORTED;
    if (n_pts == 0) return PAM_OK;
    if (!d_pts || !d_out || !d_workspace) return PAM_ERR_INVALID_ARG;
    if (workspace_bytes < eval_workspace_bytes(g->S, n_pts)) return PAM_ERR_WORKSPACE;
    return PAM_OK;
}

pam_status pam_eval(const pam_problem *prob, const pam_plan *plan, const pam_model *model,
                    const double *d_pts, int64_t n_pts, double *d_out, int log_space, int precision,
                    void *d_workspace, size_t workspace_bytes, void *stream) {
    Geo g;
    pam_status st = eval_args(prob, plan, model, true, d_pts, n_pts, d_out, precision, d_workspace,
                              workspace_bytes, &g);
    if (st != PAM_OK || n_pts == 0) return st;
    launch_eval(g, model->boxes, model->centres, model->beta, model->info, d_pts, n_pts, d_out,
                log_space, precision, d_workspace, (cudaStream_t)stream);
    PAM_CUDA_TRY(cudaGetLastError());
    return PAM_OK;
}

pam_status pam_eval_bucket(const pam_problem *prob, const pam_plan *plan, const double *d_pts, int64_t n_pts,
                           double *d_out, void *d_workspace, size_t workspace_bytes, void *stream) {
    Geo g;
    pam_status st = eval_args(prob, plan, nullptr, false, d_pts, n_pts, d_out, PAM_PREC_FP64, d_workspace,
                              workspace_bytes, &g);
    if (st != PAM_OK || n_pts == 0) return st;
    launch_eval_bucket(g, d_pts, n_pts, d_out, d_workspace, (cudaStream_t)stream);
    PAM_CUDA_TRY(cudaGetLastError());
    return PAM_OK;
}

pam_status pam_eval_bucketed(const pam_problem *prob, const pam_plan *plan, const pam_model *model,
                             const double *d_pts, int64_t n_pts, double *d_out, int log_space, int precision,
                             void *d_workspace, size_t workspace_bytes, void *stream) {
    Geo g;
    pam_status st = eval_args(prob, plan, model, true, d_pts, n_pts, d_out, precision, d_workspace,
                              workspace_bytes, &g);
    if (st != PAM_OK || n_pts == 0) return st;
    launch_eval_bucketed(g, model->boxes, model->centres, model->beta, model->info, d_pts, n_pts, d_out,
                         log_space, precision, d_workspace, (cudaStream_t)stream);
    PAM_CUDA_TRY(cudaGetLastError());
    return PAM_OK;
}

// Largest band (in cells) the glued evaluation accepts: half the narrowest
// core along every axis that has an interior face.
static double glue_band_limit(const Geo &g) {
    double lim = INFINITY;
    for (int a = 0; a < g.dim; ++a) {
        if (g.p[a] < 2) continue;
        for (int j = 0; j < g.p[a]; ++j) {
            int64_t lo = ((int64_t)j * g.n[a]) / g.p[a], hi = ((int64_t)(j + 1) * g.n[a]) / g.p[a];
            lim = fmin(lim, 0.5 * (double)(hi - lo));
        }
    }
    return lim;
}

pam_status pam_eval_glued_workspace_size(const pam_problem *prob, const pam_plan *plan, int64_t n_pts,
                                         size_t *bytes) {
    Geo g;
    pam_status st;
    if (!make_geo(prob, nullptr, &g, nullptr, &st)) return st;
    if (!plan || !bytes || n_pts < 0 || plan->n_subdomains != g.S) return PAM_ERR_INVALID_ARG;
    if (n_pts > ((int64_t)INT32_MAX >> g.dim)) return PAM_ERR_UNSUPPORTED;
    *bytes = glue_workspace_bytes(g.S, g.dim, n_pts);
    return PAM_OK;
}

pam_status pam_eval_glued(const pam_problem *prob, const pam_plan *plan, const pam_model *model,
                          const double *d_pts, int64_t n_pts, double band, double *d_out, int log_space,
                          int precision, void *d_workspace, size_t workspace_bytes, void *stream) {
    Geo g;
    pam_status st;
    if (!make_geo(prob, nullptr, &g, nullptr, &st)) return st;
    if (!plan || plan->n_subdomains != g.S || plan->m_cap > PAM_MAX_M || plan->m_cap < 1)
        return PAM_ERR_INVALID_ARG;
    g.m_cap = plan->m_cap;
    g.n_max = plan->max_patch_cells;
    if (n_pts < 0 || !model_ok(model)) return PAM_ERR_INVALID_ARG;
    if (precision != PAM_PREC_FP64 && precision != PAM_PREC_MIXED) return PAM_ERR_INVALID_ARG;
    if (!(band > 0.0) || !std::isfinite(band) || band > glue_band_limit(g)) return PAM_ERR_INVALID_ARG;
    if (n_pts > ((int64_t)INT32_MAX >> g.dim)) return PAM_ERR_UNSUPPORTED;
    if (n_pts == 0) return PAM_OK;
    if (!d_pts || !d_out || !d_workspace) return PAM_ERR_INVALID_ARG;
    if (workspace_bytes < glue_workspace_bytes(g.S, g.dim, n_pts)) return PAM_ERR_WORKSPACE;
    launch_eval_glued(g, model->boxes, model->centres, model->beta, model->info, d_pts, n_pts, band, d_out,
                      log_space, precision, d_workspace, (cudaStream_t)stream);
    PAM_CUDA_TRY(cudaGetLastError());
    return PAM_OK;
}

pam_status pam_errors(const pam_problem *prob, const pam_plan *plan, const pam_model *model,
                      const double *d_K, double *d_err, int precision, int quad, void *d_workspace,
                      size_t workspace_bytes, void *stream) {
    Geo g;
    pam_status st;
    if (!make_geo(prob, nullptr, &g, nullptr, &st)) return st;
    if (!plan || plan->n_subdomains != g.S || plan->m_cap > PAM_MAX_M || plan->m_cap < 1)
        return PAM_ERR_INVALID_ARG;
    g.m_cap = plan->m_cap;
    g.n_max = plan->max_patch_cells;
    if (!model_ok(model) || !d_K || !d_err || !d_workspace) return PAM_ERR_INVALID_ARG;
    if (precision != PAM_PREC_FP64 && precision != PAM_PREC_MIXED) return PAM_ERR_INVALID_ARG;
    if (quad != 0 && quad != 1) return PAM_ERR_INVALID_ARG;
    Ws w = carve_workspace(g, d_workspace);
    if (workspace_bytes < (size_t)((char *)w.y - (char *)d_workspace)) return PAM_ERR_WORKSPACE;
    launch_errors(g, model->boxes, model->centres, model->beta, model->info, d_K, d_err, precision,
                  quad, w, (cudaStream_t)stream);
    PAM_CUDA_TRY(cudaGetLastError());
    return PAM_OK;
}

pam_status pam_error_sums(const pam_problem *prob, const pam_plan *plan, const pam_model *model,
                          const double *d_K, double *d_sums, int precision, int quad, int sub_begin,
                          int sub_end, void *d_workspace, size_t workspace_bytes, void *stream) {
    Geo g;
    pam_status st;
    if (!make_geo(prob, nullptr, &g, nullptr, &st)) return st;
    if (!plan || plan->n_subdomains != g.S || plan->m_cap > PAM_MAX_M || plan->m_cap < 1)
        return PAM_ERR_INVALID_ARG;
    if (sub_begin < 0 || sub_end < sub_begin || sub_end > g.S) return PAM_ERR_INVALID_ARG;
    g.m_cap = plan->m_cap;
    g.n_max = plan->max_patch_cells;
    if (!model_ok(model) || !d_K || !d_sums || !d_workspace) return PAM_ERR_INVALID_ARG;
    if (precision != PAM_PREC_FP64 && precision != PAM_PREC_MIXED) return PAM_ERR_INVALID_ARG;
    if (quad != 0 && quad != 1) return PAM_ERR_INVALID_ARG;
    Ws w = carve_workspace(g, d_workspace);
    if (workspace_bytes < (size_t)((char *)w.y - (char *)d_workspace)) return PAM_ERR_WORKSPACE;
    launch_errors(g, model->boxes, model->centres, model->beta, model->info, d_K, d_sums, precision,
                  quad, w, (cudaStream_t)stream, sub_begin, sub_end);
    PAM_CUDA_TRY(cudaGetLastError());
    return PAM_OK;
}

// ------------------------------------------------------ element lists ---

// Range of cores j along one axis whose patch [lo_j - ov, hi_j + ov)
// (clipped to [0, n], closed at n) holds the cell coordinate u.
static void patch_range(int n, int p, int ov, double u, int *j0, int *j1) {
    *j0 = p;
    *j1 = -1;
    for (int j = 0; j < p; ++j) {
        int64_t lo = ((int64_t)j * n) / p - ov, hi = ((int64_t)(j + 1) * n) / p + ov;
        if (lo < 0) lo = 0;
        if (hi > n) hi = n;
        const bool in = u >= (double)lo && (hi == n ? u <= (double)hi : u < (double)hi);
        if (in) {
            if (j < *j0) *j0 = j;
            *j1 = j;
        }
    }
}

pam_status pam_partition_cells(const pam_problem *prob, const double *h_x, int64_t n_cells,
                               int32_t *h_patch_start, int32_t *h_patch_cells) {
    Geo g;
    pam_status st;
    if (!make_geo(prob, nullptr, &g, nullptr, &st)) return st;
    if (!h_patch_start || n_cells < 0 || (n_cells > 0 && !h_x)) return PAM_ERR_INVALID_ARG;
    if (n_cells > (int64_t)INT32_MAX) return PAM_ERR_UNSUPPORTED;
    std::vector<int64_t> cnt((size_t)g.S, 0);
    std::vector<int> rng((size_t)n_cells * 6);
    for (int64_t e = 0; e < n_cells; ++e) {
        int *r = &rng[(size_t)e * 6];
        for (int a = 0; a < 3; ++a) {
            r[2 * a] = 0;
            r[2 * a + 1] = 0;
        }
        for (int a = 0; a < g.dim; ++a) {
            const double xa = h_x[e * g.dim + a];
            const double u = xa * (double)g.nmax;
            if (!(u >= 0.0) || u > (double)g.n[a]) return PAM_ERR_INVALID_ARG;  // outside the domain
            patch_range(g.n[a], g.p[a], g.overlap, u, &r[2 * a], &r[2 * a + 1]);
            if (r[2 * a] > r[2 * a + 1]) return PAM_ERR_INVALID_ARG;
        }
        for (int k = r[4]; k <= r[5]; ++k)
            for (int j = r[2]; j <= r[3]; ++j)
                for (int i = r[0]; i <= r[1]; ++i) ++cnt[(size_t)(i + g.p[0] * (j + g.p[1] * k))];
    }
    int64_t run = 0;
    for (int s = 0; s < g.S; ++s) {
        h_patch_start[s] = (int32_t)run;
        run += cnt[(size_t)s];
        if (run > (int64_t)INT32_MAX) return PAM_ERR_UNSUPPORTED;
    }
    h_patch_start[g.S] = (int32_t)run;
    if (!h_patch_cells) return PAM_OK;
    std::vector<int64_t> fill((size_t)g.S, 0);
    for (int64_t e = 0; e < n_cells; ++e) {  // ascending element index within each patch
        const int *r = &rng[(size_t)e * 6];
        for (int k = r[4]; k <= r[5]; ++k)
            for (int j = r[2]; j <= r[3]; ++j)
                for (int i = r[0]; i <= r[1]; ++i) {
                    const int s = i + g.p[0] * (j + g.p[1] * k);
                    h_patch_cells[h_patch_start[s] + fill[(size_t)s]++] = (int32_t)e;
                }
    }
    return PAM_OK;
}

// Geometry of an element-list problem: the grid view, then the patch size
// from the patch lists (rounded to 32) in place of the grid patches'.
static bool geo_cells(const pam_problem *prob, const pam_params *par, int max_patch, Geo *g, Par *p,
                      pam_status *st) {
    if (!make_geo(prob, par, g, p, st)) return false;
    *st = PAM_ERR_INVALID_ARG;
    if (max_patch < 1 || max_patch > (1 << 20)) {
        *st = max_patch > (1 << 20) ? PAM_ERR_UNSUPPORTED : PAM_ERR_INVALID_ARG;
        return false;
    }
    g->n_max = (int)align_up((size_t)max_patch, 32);
    if (par && par->levels > 0) {
        int64_t P = 1;
        while (P < g->n_max) P <<= 1;
        if (P * 8 > 227 * 1024) { *st = PAM_ERR_UNSUPPORTED; return false; }
    }
    if (par && par->quad != 0) { *st = PAM_ERR_UNSUPPORTED; return false; }  // element shapes not given
    g->cells = 1;
    *st = PAM_OK;
    return true;
}

pam_status pam_plan_create_cells(const pam_problem *prob, const pam_params *par, int64_t n_cells,
                                 const int32_t *h_patch_start, pam_plan *out) {
    if (!prob || !par || !out || !h_patch_start || n_cells < 0) return PAM_ERR_INVALID_ARG;
    Geo g0;
    pam_status st;
    if (!make_geo(prob, nullptr, &g0, nullptr, &st)) return st;
    int max_patch = 0;
    for (int s = 0; s < g0.S; ++s) {
        const int32_t c = h_patch_start[s + 1] - h_patch_start[s];
        if (c < 0 || h_patch_start[s] < 0) return PAM_ERR_INVALID_ARG;
        if (c > max_patch) max_patch = c;
    }
    Geo g;
    Par p;
    if (!geo_cells(prob, par, max_patch < 1 ? 1 : max_patch, &g, &p, &st)) return st;
    Ws w;
    out->n_subdomains = g.S;
    out->max_patch_cells = g.n_max;
    out->m0 = g.m0;
    out->m_cap = g.m_cap;
    out->n_grid_cells = n_cells;
    out->workspace_bytes = carve(g, nullptr, &w);
    return PAM_OK;
}

static pam_status cells_setup(const pam_problem *prob, const pam_params *par, const pam_plan *plan,
                              const pam_cells *cells, Geo *g, Par *p) {
    pam_status st;
    if (!plan || !cells || !cells->x || !cells->vol || !cells->patch_start || !cells->patch_cells)
        return PAM_ERR_INVALID_ARG;
    if (cells->n_cells < 0 || cells->n_cells != plan->n_grid_cells) return PAM_ERR_INVALID_ARG;
    if (!geo_cells(prob, par, plan->max_patch_cells, g, p, &st)) return st;
    if (plan->n_subdomains != g->S || plan->max_patch_cells != g->n_max || plan->m_cap > PAM_MAX_M ||
        plan->m_cap < 1 || plan->m_cap % 64 != 0 || (par && plan->m_cap < g->m_cap))
        return PAM_ERR_INVALID_ARG;
    g->m_cap = plan->m_cap;
    g->cx = cells->x;
    g->cvol = cells->vol;
    g->pstart = cells->patch_start;
    g->pcells = cells->patch_cells;
    return PAM_OK;
}

pam_status pam_fit_cells(const pam_problem *prob, const pam_params *par, const pam_plan *plan,
                         const pam_cells *cells, const double *d_K, pam_model *model, void *d_workspace,
                         size_t workspace_bytes, void *stream) {
    Geo g;
    Par p;
    pam_status st;
    if (!par) return PAM_ERR_INVALID_ARG;
    if ((st = cells_setup(prob, par, plan, cells, &g, &p)) != PAM_OK) return st;
    if (par->precision == PAM_PREC_MIXED && (g.m_cap > kMixedMaxM || !mixed_solve_fits(g)))
        return PAM_ERR_UNSUPPORTED;
    if (!d_K || !model_ok(model) || !d_workspace) return PAM_ERR_INVALID_ARG;
    Ws w = carve_workspace(g, d_workspace);
    if (workspace_bytes < w.bytes) return PAM_ERR_WORKSPACE;
    g.cxv = w.cxv;
    return fit_launches(g, p, par, d_K, model, w, (cudaStream_t)stream);
}

pam_status pam_refine_cells(const pam_problem *prob, const pam_params *par, const pam_plan *plan,
                            const pam_cells *cells, const double *d_K, pam_model *model, int n_levels,
                            void *d_workspace, size_t workspace_bytes, void *stream) {
    Geo g;
    Par p;
    pam_status st;
    if (!par) return PAM_ERR_INVALID_ARG;
    if ((st = cells_setup(prob, par, plan, cells, &g, &p)) != PAM_OK) return st;
    if (par->precision == PAM_PREC_MIXED && (g.m_cap > kMixedMaxM || !mixed_solve_fits(g)))
        return PAM_ERR_UNSUPPORTED;
    if (!d_K || !model_ok(model) || !d_workspace || n_levels < 0) return PAM_ERR_INVALID_ARG;
    Ws w = carve_workspace(g, d_workspace);
    if (workspace_bytes < w.bytes) return PAM_ERR_WORKSPACE;
    g.cxv = w.cxv;
    return refine_launches(g, p, par, model, n_levels, w, (cudaStream_t)stream);
}

pam_status pam_errors_cells(const pam_problem *prob, const pam_plan *plan, const pam_model *model,
                            const pam_cells *cells, const double *d_K, double *d_err, int precision,
                            void *d_workspace, size_t workspace_bytes, void *stream) {
    Geo g;
    Par p;
    pam_status st;
    if ((st = cells_setup(prob, nullptr, plan, cells, &g, &p)) != PAM_OK) return st;
    if (!model_ok(model) || !d_K || !d_err || !d_workspace) return PAM_ERR_INVALID_ARG;
    if (precision != PAM_PREC_FP64 && precision != PAM_PREC_MIXED) return PAM_ERR_INVALID_ARG;
    Ws w = carve_workspace(g, d_workspace);
    if (workspace_bytes < (size_t)((char *)w.y - (char *)d_workspace)) return PAM_ERR_WORKSPACE;
    launch_errors_cells(g, model->boxes, model->centres, model->beta, model->info, d_K, d_err, precision, w,
                        (cudaStream_t)stream);
    PAM_CUDA_TRY(cudaGetLastError());
    return PAM_OK;
}

// ------------------------------------------------ checkpoint / resume ---

namespace {
struct ModelBlobHeader {
    char magic[8];      // "PAMMODEL"
    int32_t version;    // 1
    int32_t dim;
    int32_t n_cells[3];
    int32_t n_sub[3];
    int32_t overlap;
    int32_t g_init[3];
    int32_t n_subdomains;
    int32_t m_cap;
    int32_t reserved[4];
};
const char kBlobMagic[8] = {'P', 'A', 'M', 'M', 'O', 'D', 'E', 'L'};

size_t blob_bytes(int S, int m_cap) {
    return sizeof(ModelBlobHeader) + (size_t)S * 12 * sizeof(int32_t) + (size_t)S * m_cap * 4 * sizeof(double) +
           (size_t)S * m_cap * sizeof(double) + (size_t)S * PAM_INFO_N * sizeof(int32_t);
}

pam_status blob_geometry(const pam_problem *prob, const pam_plan *plan, Geo *g) {
    pam_status st;
    if (!make_geo(prob, nullptr, g, nullptr, &st)) return st;
    if (!plan || plan->n_subdomains != g->S || plan->m_cap < 1 || plan->m_cap > PAM_MAX_M ||
        plan->m_cap % 64 != 0)
        return PAM_ERR_INVALID_ARG;
    return PAM_OK;
}
}  // namespace

pam_status pam_model_save(const pam_problem *prob, const pam_plan *plan, const pam_model *model, void *h_buf,
                          size_t *size, void *stream) {
    Geo g;
    pam_status st;
    if (!size) return PAM_ERR_INVALID_ARG;
    if ((st = blob_geometry(prob, plan, &g)) != PAM_OK) return st;
    const size_t need = blob_bytes(g.S, plan->m_cap);
    if (!h_buf) {
        *size = need;
        return PAM_OK;
    }
    if (*size < need) {
        *size = need;
        return PAM_ERR_INVALID_ARG;
    }
    if (!model_ok(model)) return PAM_ERR_INVALID_ARG;
    ModelBlobHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kBlobMagic, 8);
    h.version = 1;
    h.dim = prob->dim;
    for (int a = 0; a < 3; ++a) {
        h.n_cells[a] = g.n[a];
        h.n_sub[a] = g.p[a];
        h.g_init[a] = g.g[a];
    }
    h.overlap = g.overlap;
    h.n_subdomains = g.S;
    h.m_cap = plan->m_cap;
    char *b = (char *)h_buf;
    memcpy(b, &h, sizeof(h));
    size_t off = sizeof(h);
    const size_t S = (size_t)g.S, mc = (size_t)plan->m_cap;
    cudaStream_t st_ = (cudaStream_t)stream;
    PAM_CUDA_TRY(cudaMemcpyAsync(b + off, model->boxes, S * 12 * 4, cudaMemcpyDeviceToHost, st_));
    off += S * 12 * 4;
    PAM_CUDA_TRY(cudaMemcpyAsync(b + off, model->centres, S * mc * 4 * 8, cudaMemcpyDeviceToHost, st_));
    off += S * mc * 4 * 8;
    PAM_CUDA_TRY(cudaMemcpyAsync(b + off, model->beta, S * mc * 8, cudaMemcpyDeviceToHost, st_));
    off += S * mc * 8;
    PAM_CUDA_TRY(cudaMemcpyAsync(b + off, model->info, S * PAM_INFO_N * 4, cudaMemcpyDeviceToHost, st_));
    PAM_CUDA_TRY(cudaStreamSynchronize(st_));
    *size = need;
    return PAM_OK;
}

pam_status pam_model_load(const pam_problem *prob, const pam_plan *plan, const void *h_buf, size_t size,
                          pam_model *model, void *stream) {
    Geo g;
    pam_status st;
    if ((st = blob_geometry(prob, plan, &g)) != PAM_OK) return st;
    if (!h_buf || !model_ok(model)) return PAM_ERR_INVALID_ARG;
    const size_t need = blob_bytes(g.S, plan->m_cap);
    if (size < need) return PAM_ERR_INVALID_ARG;
    ModelBlobHeader h;
    memcpy(&h, h_buf, sizeof(h));
    if (memcmp(h.magic, kBlobMagic, 8) != 0 || h.version != 1 || h.dim != prob->dim || h.overlap != g.overlap ||
        h.n_subdomains != g.S || h.m_cap != plan->m_cap)
        return PAM_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (h.n_cells[a] != g.n[a] || h.n_sub[a] != g.p[a] || h.g_init[a] != g.g[a]) return PAM_ERR_INVALID_ARG;
    const char *b = (const char *)h_buf;
    const size_t S = (size_t)g.S, mc = (size_t)plan->m_cap;
    // the boxes must be this problem's partition, and every size within the capacity
    std::vector<int32_t> boxes(S * 12);
    if ((st = pam_partition(prob, boxes.data())) != PAM_OK) return st;
    if (memcmp(boxes.data(), b + sizeof(h), S * 12 * 4) != 0) return PAM_ERR_INVALID_ARG;
    const char *info = b + sizeof(h) + S * 12 * 4 + S * mc * 40;
    for (size_t s = 0; s < S; ++s) {
        int32_t m;
        memcpy(&m, info + (s * PAM_INFO_N + PAM_INFO_M) * sizeof(int32_t), sizeof(m));  // any alignment
        if (m < 1 || m > (int32_t)mc) return PAM_ERR_INVALID_ARG;
    }
    cudaStream_t st_ = (cudaStream_t)stream;
    size_t off = sizeof(h);
    PAM_CUDA_TRY(cudaMemcpyAsync(model->boxes, b + off, S * 12 * 4, cudaMemcpyHostToDevice, st_));
    off += S * 12 * 4;
    PAM_CUDA_TRY(cudaMemcpyAsync(model->centres, b + off, S * mc * 4 * 8, cudaMemcpyHostToDevice, st_));
    off += S * mc * 4 * 8;
    PAM_CUDA_TRY(cudaMemcpyAsync(model->beta, b + off, S * mc * 8, cudaMemcpyHostToDevice, st_));
    off += S * mc * 8;
    PAM_CUDA_TRY(cudaMemcpyAsync(model->info, b + off, S * PAM_INFO_N * 4, cudaMemcpyHostToDevice, st_));
    PAM_CUDA_TRY(cudaStreamSynchronize(st_));
    return PAM_OK;
}

// Data preparation and one solve of every running subdomain from the
// model's coefficients: afterwards the workspace holds what pam_refine
// reads (cell data, indicators of the current coefficients).
static pam_status resume_launches(const Geo &g, const Par &p, const pam_params *par, const double *d_K,
                                  pam_model *model, const Ws &w, cudaStream_t s) {
    pam_status st;
    const bool deferred = par->deferred_status != 0;
    PAM_CUDA_TRY(cudaMemsetAsync(w.status, 0, 8 * sizeof(int32_t), s));
    launch_prepare(g, model->boxes, d_K, w, s);
    PAM_CUDA_TRY(cudaGetLastError());
    int32_t hs[8];
    if (!deferred) {
        if ((st = read_status(w, s, hs)) != PAM_OK) return st;
        if (hs[kStBadK]) return PAM_ERR_NONPOSITIVE_K;
    }
    if (par->precision == PAM_PREC_MIXED)
        launch_solve_level_mixed(g, p, model->boxes, model->centres, model->beta, model->info, w, s);
    else
        launch_solve_level_f64(g, p, model->boxes, model->centres, model->beta, model->info, w, s);
    PAM_CUDA_TRY(cudaGetLastError());
    if (deferred) return PAM_OK;
    if ((st = read_status(w, s, hs)) != PAM_OK) return st;
    if (hs[kStTimeout]) return PAM_ERR_TIMEOUT;
    return hs[kStUncertified] ? PAM_ERR_NOT_CONVERGED : PAM_OK;
}

pam_status pam_resume(const pam_problem *prob, const pam_params *par, const pam_plan *plan, const double *d_K,
                      pam_model *model, void *d_workspace, size_t workspace_bytes, void *stream) {
    Geo g;
    Par p;
    pam_status st;
    if (!par || !make_geo(prob, par, &g, &p, &st)) return par ? st : PAM_ERR_INVALID_ARG;
    if ((st = check_plan(g, plan)) != PAM_OK) return st;
    g.m_cap = plan->m_cap;
    if (par->precision == PAM_PREC_MIXED && (g.m_cap > kMixedMaxM || !mixed_solve_fits(g)))
        return PAM_ERR_UNSUPPORTED;
    if (!d_K || !model_ok(model) || !d_workspace) return PAM_ERR_INVALID_ARG;
    Ws w = carve_workspace(g, d_workspace);
    if (workspace_bytes < w.bytes) return PAM_ERR_WORKSPACE;
    return resume_launches(g, p, par, d_K, model, w, (cudaStream_t)stream);
}

pam_status pam_resume_cells(const pam_problem *prob, const pam_params *par, const pam_plan *plan,
                            const pam_cells *cells, const double *d_K, pam_model *model, void *d_workspace,
                            size_t workspace_bytes, void *stream) {
    Geo g;
    Par p;
    pam_status st;
    if (!par) return PAM_ERR_INVALID_ARG;
    if ((st = cells_setup(prob, par, plan, cells, &g, &p)) != PAM_OK) return st;
    if (par->precision == PAM_PREC_MIXED && (g.m_cap > kMixedMaxM || !mixed_solve_fits(g)))
        return PAM_ERR_UNSUPPORTED;
    if (!d_K || !model_ok(model) || !d_workspace) return PAM_ERR_INVALID_ARG;
    Ws w = carve_workspace(g, d_workspace);
    if (workspace_bytes < w.bytes) return PAM_ERR_WORKSPACE;
    g.cxv = w.cxv;
    return resume_launches(g, p, par, d_K, model, w, (cudaStream_t)stream);
}

// ---------------------------------------------------------- autotuning ---


pam_status pam_tuning_set(const pam_tuning *t) {
    if (!t) {
        memset(&g_tuning, 0, sizeof(g_tuning));
        return PAM_OK;
    }
    if (t->factor_kb < 0 || (t->factor_kb > 0 && (t->factor_kb < 4 || t->factor_kb > 200))) return PAM_ERR_INVALID_ARG;
    if (t->eval_block != 0 && t->eval_block != 128 && t->eval_block != 256 && t->eval_block != 512 &&
        t->eval_block != 1024)
        return PAM_ERR_INVALID_ARG;
    if (t->gram_stages != 0 && t->gram_stages != 2 && t->gram_stages != 3) return PAM_ERR_INVALID_ARG;
    if (t->solve_persistent != 0 && t->solve_persistent != 1) return PAM_ERR_INVALID_ARG;
    if (t->level_groups < 0 || t->level_groups > 2) return PAM_ERR_INVALID_ARG;
    g_tuning = *t;
    return PAM_OK;
}

int pam_group_layout(int n_subdomains, int32_t *out) {
    if (n_subdomains < 1 || !out) return -1;
    Geo g{};
    g.S = n_subdomains;
    pam_params par{};
    par.precision = PAM_PREC_MIXED;
    Ws w{};
    w.fb_slots = n_subdomains < kFbSlots ? n_subdomains : kFbSlots;
    const int ng = level_groups(g, &par, w, false);
    for (int q = 0; q < ng; ++q) {
        const GroupLayout l = group_layout(g.S, w.fb_slots, q, ng);
        const int32_t v[7] = {l.gb, l.gs, l.gn, l.order_off, l.list_off, l.slots, l.slot0};
        for (int k = 0; k < 7; ++k) out[7 * q + k] = v[k];
    }
    return ng;
}

pam_status pam_tuning_get(pam_tuning *t) {
    if (!t) return PAM_ERR_INVALID_ARG;
    *t = g_tuning;
    return PAM_OK;
}

// A candidate replaces the one kept so far (the built-in first) only when
// it measures at least 2 % faster: the medians of three runs differ by about
// 1 % between equivalent launches, and a choice made on noise would move
// the step from run to run.
constexpr double kTuneMargin = 0.98;

static pam_status autotune_run(Geo g, const Par &p, const pam_params *par, pam_model *model, const Ws &w,
                               const double *d_pts, int64_t n_pts, double *d_out, void *d_eval_workspace,
                               cudaStream_t s, pam_tuning *out, double *h_ms) {
    pam_status st;
    const bool mixed = par->precision == PAM_PREC_MIXED;
    if (mixed && (g.m_cap > kMixedMaxM || !mixed_solve_fits(g))) return PAM_ERR_UNSUPPORTED;
    if (h_ms)
        for (int i = 0; i < 14; ++i) h_ms[i] = -1.0;
    const pam_tuning keep = g_tuning;
    pam_tuning best = g_tuning;
    double t;
    PAM_CUDA_TRY(cudaMemsetAsync(w.status, 0, 8 * sizeof(int32_t), s));
    if (mixed) {
        // the tensor-core Gram's pipeline depth (3 stages only where they fit)
        const int gst[2] = {3, 2};
        double bt = INFINITY;
        for (int i = 0; i < 2; ++i) {
            g_tuning.gram_stages = gst[i];
            if ((st = time_median(s, [&] { launch_stats_gram_tc(g, model->boxes, model->centres, model->info, w, s, 1); },
                                  &t)) != PAM_OK) { g_tuning = keep; return st; }
            if (h_ms) h_ms[i] = t;
            if (i == 0 || t < kTuneMargin * bt) { bt = t; best.gram_stages = gst[i]; }
        }
        g_tuning.gram_stages = best.gram_stages;
        // the solve's shared-memory factor budget (0: the built-in choice);
        // every subdomain is re-solved from its coefficients (same minimiser)
        const int fkb[6] = {0, 64, 48, 32, 24, 16};
        bt = INFINITY;
        for (int i = 0; i < 6; ++i) {
            g_tuning.factor_kb = fkb[i];
            if (!mixed_solve_fits(g)) continue;
            if ((st = time_median(s, [&] {
                     launch_solve_mixed(g, p, model->boxes, model->centres, model->beta, model->info, w, nullptr, 1,
                                        nullptr, 0, s, 1);
                 }, &t)) != PAM_OK) { g_tuning = keep; return st; }
            if (h_ms) h_ms[2 + i] = t;
            if (i == 0 || t < kTuneMargin * bt) { bt = t; best.factor_kb = fkb[i]; }
        }
        g_tuning.factor_kb = best.factor_kb;
    }
    if (n_pts > 0) {
        // the evaluation's threads per block (model and points as given)
        const int eb[4] = {128, 256, 512, 1024};
        double te[4];
        for (int i = 0; i < 4; ++i) {
            g_tuning.eval_block = eb[i];
            if ((st = time_median(s, [&] {
                     launch_eval(g, model->boxes, model->centres, model->beta, model->info, d_pts, n_pts, d_out, 0,
                                 par->precision, d_eval_workspace, s);
                 }, &te[i])) != PAM_OK) { g_tuning = keep; return st; }
            if (h_ms) h_ms[8 + i] = te[i];
        }
        // the built-in 256 unless another size is 2 % faster
        double bt = te[1];
        best.eval_block = 0;
        for (int i = 0; i < 4; ++i)
            if (i != 1 && te[i] < kTuneMargin * te[1] && te[i] < bt) { bt = te[i]; best.eval_block = eb[i]; }
    }
    if (mixed) {
        // the solve's launch: one CTA per subdomain, or resident CTAs taking
        // subdomains from a counter (same order, same results)
        double bt = INFINITY;
        for (int i = 0; i < 2; ++i) {
            g_tuning.solve_persistent = i;
            if ((st = time_median(s, [&] {
                     launch_solve_mixed(g, p, model->boxes, model->centres, model->beta, model->info, w, nullptr, 1,
                                        nullptr, 0, s, 1);
                 }, &t)) != PAM_OK) { g_tuning = keep; return st; }
            if (h_ms) h_ms[12 + i] = t;
            if (i == 0 || t < kTuneMargin * bt) { bt = t; best.solve_persistent = i; }
        }
    }
    g_tuning = best;
    *out = best;
    int32_t hs[8];
    if ((st = read_status(w, s, hs)) != PAM_OK) return st;
    if (hs[kStTimeout]) return PAM_ERR_TIMEOUT;
    return PAM_OK;
}

pam_status pam_autotune(const pam_problem *prob, const pam_params *par, const pam_plan *plan, const double *d_K,
                        pam_model *model, void *d_workspace, size_t workspace_bytes, const double *d_pts,
                        int64_t n_pts, double *d_out, void *d_eval_workspace, size_t eval_ws_bytes,
                        void *stream, pam_tuning *out, double *h_ms) {
    Geo g;
    Par p;
    pam_status st;
    if (!par || !make_geo(prob, par, &g, &p, &st)) return par ? st : PAM_ERR_INVALID_ARG;
    if ((st = check_plan(g, plan)) != PAM_OK) return st;
    g.m_cap = plan->m_cap;
    if (!d_K || !model_ok(model) || !d_workspace || !out || n_pts < 0) return PAM_ERR_INVALID_ARG;
    if (n_pts > 0 && (!d_pts || !d_out || !d_eval_workspace)) return PAM_ERR_INVALID_ARG;
    if (n_pts > (int64_t)INT32_MAX) return PAM_ERR_UNSUPPORTED;
    if (n_pts > 0 && eval_ws_bytes < eval_workspace_bytes(g.S, n_pts)) return PAM_ERR_WORKSPACE;
    Ws w = carve_workspace(g, d_workspace);
    if (workspace_bytes < w.bytes) return PAM_ERR_WORKSPACE;
    return autotune_run(g, p, par, model, w, d_pts, n_pts, d_out, d_eval_workspace, (cudaStream_t)stream, out,
                        h_ms);
}

pam_status pam_autotune_cells(const pam_problem *prob, const pam_params *par, const pam_plan *plan,
                              const pam_cells *cells, const double *d_K, pam_model *model, void *d_workspace,
                              size_t workspace_bytes, const double *d_pts, int64_t n_pts, double *d_out,
                              void *d_eval_workspace, size_t eval_ws_bytes, void *stream, pam_tuning *out,
                              double *h_ms) {
    Geo g;
    Par p;
    pam_status st;
    if (!par) return PAM_ERR_INVALID_ARG;
    if ((st = cells_setup(prob, par, plan, cells, &g, &p)) != PAM_OK) return st;
    if (!d_K || !model_ok(model) || !d_workspace || !out || n_pts < 0) return PAM_ERR_INVALID_ARG;
    if (n_pts > 0 && (!d_pts || !d_out || !d_eval_workspace)) return PAM_ERR_INVALID_ARG;
    if (n_pts > (int64_t)INT32_MAX) return PAM_ERR_UNSUPPORTED;
    if (n_pts > 0 && eval_ws_bytes < eval_workspace_bytes(g.S, n_pts)) return PAM_ERR_WORKSPACE;
    Ws w = carve_workspace(g, d_workspace);
    if (workspace_bytes < w.bytes) return PAM_ERR_WORKSPACE;
    g.cxv = w.cxv;
    return autotune_run(g, p, par, model, w, d_pts, n_pts, d_out, d_eval_workspace, (cudaStream_t)stream, out,
                        h_ms);
}

pam_status pam_selftest_wait(int arrive, long long budget_cycles, int32_t *d_flag, void *stream) {
    if ((arrive != 0 && arrive != 1) || budget_cycles < 1000 || budget_cycles > 4000000000LL || !d_flag)
        return PAM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    launch_wait_selftest(arrive, budget_cycles, d_flag, s);
    PAM_CUDA_TRY(cudaGetLastError());
    int32_t h = -1;
    PAM_CUDA_TRY(cudaMemcpyAsync(&h, d_flag, sizeof(h), cudaMemcpyDeviceToHost, s));
    PAM_CUDA_TRY(cudaStreamSynchronize(s));
    return h == 1 ? PAM_ERR_TIMEOUT : (h == 0 ? PAM_OK : PAM_ERR_CUDA);
}

}  // extern "C"
