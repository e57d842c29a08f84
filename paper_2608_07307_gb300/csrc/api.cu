// api.cu -- the C ABI of libsrp (include/srp.h): validation, device memory,
// mesh build and the per-batch launch sequence.  No exception crosses the ABI.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "srp_internal.cuh"

using namespace srp;

namespace {

// Evaluation chunks rotate over this many lane streams.
constexpr int kLanes = 4;

struct Mesh {
    MeshDev h{};                 // host copy holding device pointers
    MeshDev *d = nullptr;        // device copy
    std::vector<void *> allocs;  // device allocations owned by the mesh
    float4 *node_tmpl_dyn = nullptr;  // 4-wide nodes of the dynamic parts: refs, meta, empty boxes
    double *angles_d = nullptr;  // commanded angles / offsets [n_parts]
    double mass = 0.0;
    int slots = 0;
    SlotBufs sb{};
    std::vector<void *> slot_allocs;
};

}  // namespace

struct srp_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    std::vector<Mesh *> meshes;
    // workspace, grown on demand
    SlotPose *pose = nullptr;
    size_t pose_cap = 0;
    float *partials = nullptr;
    size_t partials_cap = 0;
    unsigned *pcounts = nullptr;
    size_t pcounts_cap = 0;
    int *amb_list = nullptr;
    size_t amb_list_cap = 0;
    double *partials1 = nullptr;
    size_t partials1_cap = 0;
    unsigned *red_ticket = nullptr;
    size_t red_ticket_cap = 0;
    double *dpart = nullptr;  // diffuse-ray partial sums [SL][kDiffBlocks][6]
    size_t dpart_cap = 0;
    DEmit *demit = nullptr;   // diffuse emission records [SL][R][nseg - 1]
    size_t demit_cap = 0;
    int *dcnt = nullptr;      // their counts, then prefix, per ray [SL][R]
    size_t dcnt_cap = 0;
    int *dtot = nullptr;      // per slot [SL]
    size_t dtot_cap = 0;
    unsigned char *tctx = nullptr;
    size_t tctx_cap = 0;
    int *amb_count = nullptr;
    size_t amb_count_cap = 0;
    // rasterised primary visibility: pixel buffers (kept cleared), per-lane chunk lists
    unsigned long long *pix_key = nullptr;
    size_t pix_key_cap = 0;
    unsigned *qstate = nullptr;  // work-queue state, qstate_words(S) per lane
    size_t qstate_cap = 0;
    unsigned *pix_cand = nullptr;
    size_t pix_cand_cap = 0;
    int4 *big = nullptr;
    size_t big_cap = 0;
    unsigned *big_count = nullptr;
    size_t big_count_cap = 0;
    int2 *bigt = nullptr;
    size_t bigt_cap = 0;
    unsigned *bigt_count = nullptr;
    size_t bigt_count_cap = 0;
    int *rast_bad = nullptr;
    size_t rast_bad_cap = 0;
    double *io = nullptr;
    size_t io_cap = 0;
    int32_t *hits = nullptr;
    size_t hits_cap = 0;
    int *err_flags = nullptr;
    unsigned long long *stats = nullptr;
    srp_eval_stats last{};
    std::vector<cudaEvent_t> events;  // pool for SRP_EVAL_TIMING
    // propagation
    double *prop_io = nullptr;
    size_t prop_io_cap = 0;
    double *spad_buf = nullptr;  // SPAD: sample directions and results, or a staged table
    size_t spad_cap = 0;
    PropState *prop_state = nullptr;
    size_t prop_state_cap = 0;
    double *prop_hlog = nullptr;
    size_t prop_hlog_cap = 0;
    double *prop_replay = nullptr;
    size_t prop_replay_cap = 0;
    int *prop_done = nullptr;
    // adjoint
    double *adj_partials = nullptr;
    size_t adj_partials_cap = 0;
    double *adj_partials2 = nullptr;
    size_t adj_partials2_cap = 0;
    int *win_ids = nullptr;
    size_t win_ids_cap = 0;
    double *win_val = nullptr;
    size_t win_val_cap = 0;
    int *win_pid = nullptr;
    size_t win_pid_cap = 0;
    double *gio = nullptr;
    size_t gio_cap = 0;
    // propagation adjoint
    int32_t *arc_hits = nullptr;
    size_t arc_hits_cap = 0;
    unsigned char *arc_buf = nullptr;
    size_t arc_buf_cap = 0;
    // per-slot descriptors of the current plan (device copy and the host copy it was made from)
    SlotDesc *sdesc = nullptr;
    size_t sdesc_cap = 0;
    std::vector<SlotDesc> sdesc_host;
    // autotuned trace tile width per (mesh, N, segments)
    std::map<std::tuple<const void *, int, int>, int> tile_w;
    cudaStream_t lane[kLanes] = {};  // pipeline lanes (forked from / joined to `stream`)
    cudaEvent_t ev_fork = nullptr, ev_join[kLanes] = {};
    // a side stream per lane: the refit runs beside the frame and raster passes
    cudaStream_t aux[kLanes] = {};
    cudaEvent_t ev_refit_fork[kLanes] = {}, ev_refit_join[kLanes] = {};
};

namespace {

srp_status fail(srp_ctx *ctx, srp_status code, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

#define CK(ctx, x)                                                                                   \
    do {                                                                                             \
        cudaError_t e_ = (x);                                                                        \
        if (e_ != cudaSuccess) {                                                                     \
            srp_status c_ = (e_ == cudaErrorMemoryAllocation) ? SRP_ERR_OOM : SRP_ERR_CUDA;           \
            return fail(ctx, c_, "%s failed: %s (%s:%d)", #x, cudaGetErrorString(e_), __FILE__, __LINE__); \
        }                                                                                            \
    } while (0)

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device memory of the library in this process, against an optional cap
// (srp_set_memory_limit): every allocation and release of this file goes
// through dalloc / dfree, which book the bytes.
std::mutex g_mem_mu;
size_t g_mem_limit = 0, g_mem_used = 0;
std::unordered_map<void *, size_t> g_mem_sizes;

cudaError_t dalloc_raw(void **p, size_t bytes)
{
    std::lock_guard<std::mutex> lk(g_mem_mu);
    *p = nullptr;
    if (g_mem_limit && g_mem_used + bytes > g_mem_limit) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return e;
    g_mem_used += bytes;
    g_mem_sizes[*p] = bytes;
    return cudaSuccess;
}

template <class T>
cudaError_t dalloc(T **p, size_t bytes)
{
    return dalloc_raw(reinterpret_cast<void **>(p), bytes);
}

void dfree(void *p)
{
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_mem_mu);
        auto it = g_mem_sizes.find(p);
        if (it != g_mem_sizes.end()) {
            g_mem_used -= it->second;
            g_mem_sizes.erase(it);
        }
    }
    cudaFree(p);
}

template <class T>
cudaError_t dmalloc(std::vector<void *> &owner, T **p, size_t count)
{
    void *q = nullptr;
    cudaError_t e = dalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    owner.push_back(q);
    *p = static_cast<T *>(q);
    return cudaSuccess;
}

template <class T>
cudaError_t grow(T **p, size_t *cap, size_t need, bool zero)
{
    if (need <= *cap) return cudaSuccess;
    if (*p) dfree(*p);
    *p = nullptr;
    *cap = 0;
    size_t n = std::max<size_t>(need, 1);
    cudaError_t e = dalloc((void **)p, n * sizeof(T));
    if (e != cudaSuccess) return e;
    if (zero) {
        e = cudaMemset(*p, 0, n * sizeof(T));
        if (e != cudaSuccess) return e;
    }
    *cap = n;
    return cudaSuccess;
}

// grow, then set every byte of a new buffer to `byte` before any later work
// on any stream can touch it.
template <class T>
cudaError_t grow_fill(T **p, size_t *cap, size_t need, int byte)
{
    if (need <= *cap) return cudaSuccess;
    cudaError_t e = grow(p, cap, need, false);
    if (e != cudaSuccess) return e;
    e = cudaMemset(*p, byte, *cap * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaDeviceSynchronize();
}

void free_mesh(Mesh *m)
{
    if (!m) return;
    for (void *p : m->slot_allocs) dfree(p);
    for (void *p : m->allocs) dfree(p);
    delete m;
}

// Allocate per-slot dynamic storage for S concurrent evaluations.
srp_status ensure_slots(srp_ctx *ctx, Mesh *m, int S)
{
    if (m->slots >= S) return SRP_OK;
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (void *p : m->slot_allocs) dfree(p);
    m->slot_allocs.clear();
    m->slots = 0;
    const MeshDev &h = m->h;
    SlotBufs &b = m->sb;
    CK(ctx, dmalloc(m->slot_allocs, &b.vert64, (size_t)S * h.n_dyn_verts * 3));
    CK(ctx, dmalloc(m->slot_allocs, &b.vview, (size_t)S * h.n_verts));
    CK(ctx, dmalloc(m->slot_allocs, &b.vview64, (size_t)S * h.n_verts * 3));
    CK(ctx, dmalloc(m->slot_allocs, &b.tri, (size_t)S * h.n_dyn_tris * 3));
    CK(ctx, dmalloc(m->slot_allocs, &b.node, (size_t)S * h.n_dyn_nodes * kNode4));
    CK(ctx, dmalloc(m->slot_allocs, &b.counter, (size_t)S * h.n_dyn_nodes));
    CK(ctx, dmalloc(m->slot_allocs, &b.root_box, (size_t)S * kMaxParts * 6));
    CK(ctx, cudaMemset(b.counter, 0, sizeof(unsigned) * std::max<size_t>((size_t)S * h.n_dyn_nodes, 1)));
    CK(ctx, cudaMemset(b.root_box, 0, sizeof(float) * (size_t)S * kMaxParts * 6));
    for (int s = 0; s < S && h.n_dyn_nodes > 0; s++) {
        // child refs, links and empty boxes of the dynamic nodes (the refit fills the used boxes)
        CK(ctx, cudaMemcpy(b.node + (size_t)s * h.n_dyn_nodes * kNode4, m->node_tmpl_dyn,
                           sizeof(float4) * kNode4 * h.n_dyn_nodes, cudaMemcpyDeviceToDevice));
    }
    m->slots = S;
    return SRP_OK;
}

constexpr int kGroupMin = 64;  // smallest coplanar group given a subtree of its own

// Coplanar groups of one part, rest pose, FP64: triangles whose three vertices
// lie within 1e-13 of the part's extent of one plane.  Candidates share a
// quantised plane (unit normal with its largest component positive, offset);
// each group is then checked against its first triangle's plane.  Writes the
// group number (1, 2, ...; 0 = none) of each triangle into tgrp and the group's
// largest vertex deviation (metres) into tdev.  A ray leaving a plane meets no
// triangle lying in it, so a reflected ray may skip its origin's group.
void coplanar_groups(const std::vector<int> &tris, const int *tri, const std::vector<double> &xyz, double ext,
                     std::vector<int> &tgrp, std::vector<double> &tdev)
{
    ext = std::max(ext, 1e-300);
    const double tol = 1e-13 * ext;
    auto plane = [&](int t, double *n, double &d) {
        const double *a = &xyz[3 * (size_t)tri[3 * t]], *b = &xyz[3 * (size_t)tri[3 * t + 1]],
                     *c = &xyz[3 * (size_t)tri[3 * t + 2]];
        double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        n[0] = e1[1] * e2[2] - e1[2] * e2[1];
        n[1] = e1[2] * e2[0] - e1[0] * e2[2];
        n[2] = e1[0] * e2[1] - e1[1] * e2[0];
        double l = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        int k = 0;
        for (int q = 1; q < 3; q++) if (std::fabs(n[q]) > std::fabs(n[k])) k = q;
        if (n[k] < 0.0) l = -l;
        for (int q = 0; q < 3; q++) n[q] /= l;
        d = n[0] * a[0] + n[1] * a[1] + n[2] * a[2];
    };
    std::map<std::array<long long, 4>, std::vector<int>> bucket;
    for (int t : tris) {
        double n[3], d;
        plane(t, n, d);
        const double q = 1048576.0;
        bucket[{std::llround(n[0] * q), std::llround(n[1] * q), std::llround(n[2] * q), std::llround(d / ext * q)}]
            .push_back(t);
    }
    int g = 0;
    for (auto &kv : bucket) {
        if ((int)kv.second.size() < kGroupMin || g >= 0xffff) continue;
        double n[3], d;
        plane(kv.second[0], n, d);
        std::vector<int> keep;
        double dmax = 0.0;
        for (int t : kv.second) {
            double e = 0.0;
            for (int c = 0; c < 3; c++) {
                const double *v = &xyz[3 * (size_t)tri[3 * t + c]];
                e = std::max(e, std::fabs(n[0] * v[0] + n[1] * v[1] + n[2] * v[2] - d));
            }
            if (e <= tol) { keep.push_back(t); dmax = std::max(dmax, e); }
        }
        if ((int)keep.size() < kGroupMin) continue;
        g++;
        for (int t : keep) { tgrp[t] = g; tdev[t] = dmax; }
    }
}

// Collapse one part's binary radix tree (part-local refs: x, y children, >= 0
// internal, < 0 ~leaf) into 4-wide nodes appended to tmpl (kNode4 float4 each:
// empty child boxes, child refs, (parent, slot, children, 0)).  A node takes
// its binary node's two children and keeps splitting the internal child whose
// rest-pose box has the largest surface area until it holds four.  A binary
// node whose leaves are exactly one of the ranges in `pin` is never split into
// its parent: it heads a 4-wide node of its own, whose part-local ref goes to
// pin_ref (kEmptyChild where no binary node covers the range).  lp4 gets
// (node << 2) | slot of every leaf.  Returns the depth of the 4-wide tree.
int collapse_part(const int4 *br, int tc, int tb, const std::vector<int> &svidx, const std::vector<double> &rest,
                  const std::vector<std::pair<int, int>> &pin, std::vector<int> &pin_ref, std::vector<float4> &tmpl,
                  int *lp4)
{
    pin_ref.assign(pin.size(), kEmptyChild);
    if (tc < 2) return 0;
    const int nbin = tc - 1;
    std::vector<int> rlo(nbin), rhi(nbin), pin_of(nbin, -1);
    const double inf = std::numeric_limits<double>::infinity();
    std::vector<double> bx(6 * (size_t)nbin);
    std::vector<float> area(nbin, 0.f);
    auto child_box = [&](int ref, double *b) {
        if (ref >= 0) {
            for (int k = 0; k < 6; k++) b[k] = bx[6 * (size_t)ref + k];
            return;
        }
        for (int k = 0; k < 3; k++) { b[k] = inf; b[3 + k] = -inf; }
        for (int c = 0; c < 3; c++) {
            const double *x = &rest[3 * (size_t)svidx[3 * (size_t)(tb + ~ref) + c]];
            for (int k = 0; k < 3; k++) { b[k] = std::min(b[k], x[k]); b[3 + k] = std::max(b[3 + k], x[k]); }
        }
    };
    // rest-pose boxes of the binary nodes, children before parents
    std::vector<std::pair<int, int>> stk;
    stk.push_back({0, 0});
    while (!stk.empty()) {
        const int n = stk.back().first, state = stk.back().second;
        if (state < 2) {
            stk.back().second = state + 1;
            const int c = state == 0 ? br[n].x : br[n].y;
            if (c >= 0) stk.push_back({c, 0});
            continue;
        }
        double a[6], b[6];
        child_box(br[n].x, a);
        child_box(br[n].y, b);
        rlo[n] = std::min(br[n].x >= 0 ? rlo[br[n].x] : ~br[n].x, br[n].y >= 0 ? rlo[br[n].y] : ~br[n].y);
        rhi[n] = std::max(br[n].x >= 0 ? rhi[br[n].x] : ~br[n].x, br[n].y >= 0 ? rhi[br[n].y] : ~br[n].y);
        for (int k = 0; k < 3; k++) {
            bx[6 * (size_t)n + k] = std::min(a[k], b[k]);
            bx[6 * (size_t)n + 3 + k] = std::max(a[3 + k], b[3 + k]);
        }
        const double dx = bx[6 * (size_t)n + 3] - bx[6 * (size_t)n], dy = bx[6 * (size_t)n + 4] - bx[6 * (size_t)n + 1],
                     dz = bx[6 * (size_t)n + 5] - bx[6 * (size_t)n + 2];
        area[n] = (float)(2.0 * (dx * dy + dy * dz + dz * dx));
        stk.pop_back();
    }
    if (!pin.empty()) {
        std::map<std::pair<int, int>, int> by_range;
        for (int n = 0; n < nbin; n++) by_range[{rlo[n], rhi[n]}] = n;
        for (size_t i = 0; i < pin.size(); i++) {
            auto it = by_range.find(pin[i]);
            if (it != by_range.end()) pin_of[it->second] = (int)i;
        }
    }
    const int base = (int)(tmpl.size() / kNode4);
    const float finf = std::numeric_limits<float>::infinity();
    struct Item { int bin, parent, slot, depth; };
    std::vector<Item> todo{{0, -1, 0, 1}};
    int maxd = 0;
    while (!todo.empty()) {
        const Item it = todo.back();
        todo.pop_back();
        const int me = (int)(tmpl.size() / kNode4) - base;
        if (pin_of[it.bin] >= 0) pin_ref[pin_of[it.bin]] = me;
        int ch[4] = {br[it.bin].x, br[it.bin].y, kEmptyChild, kEmptyChild};
        int n = 2;
        while (n < 4) {
            int best = -1;
            float ba = -1.f;
            for (int k = 0; k < n; k++)
                if (ch[k] >= 0 && pin_of[ch[k]] < 0 && area[ch[k]] > ba) { ba = area[ch[k]]; best = k; }
            if (best < 0) break;
            const int c = ch[best];
            for (int k = n; k > best + 1; k--) ch[k] = ch[k - 1];
            ch[best] = br[c].x;
            ch[best + 1] = br[c].y;
            n++;
        }
        tmpl.resize(tmpl.size() + kNode4);
        float4 *nd = &tmpl[tmpl.size() - kNode4];
        for (int k = 0; k < 6; k++) {
            const float v = (k % 2 == 0) ? finf : -finf;  // lo.x hi.x lo.y hi.y lo.z hi.z: empty
            nd[k] = make_float4(v, v, v, v);
        }
        int4 refs = make_int4(ch[0], ch[1], ch[2], ch[3]), meta = make_int4(it.parent, it.slot, n, 0);
        memcpy(&nd[6], &refs, sizeof refs);
        memcpy(&nd[7], &meta, sizeof meta);
        if (it.parent >= 0) {
            int *pr = reinterpret_cast<int *>(&tmpl[(size_t)(base + it.parent) * kNode4 + 6]);
            pr[it.slot] = me;
        }
        for (int k = 0; k < n; k++) {
            if (ch[k] < 0) lp4[~ch[k]] = (me << 2) | k;
            else todo.push_back({ch[k], me, k, it.depth + 1});
        }
        maxd = std::max(maxd, it.depth);
    }
    return maxd;
}

Mesh *get_mesh(srp_ctx *ctx, int32_t id)
{
    if (!ctx || id < 0 || id >= (int32_t)ctx->meshes.size()) return nullptr;
    return ctx->meshes[id];
}


// ------------------------------------------------------------ evaluation
srp_status check_eval_params(srp_ctx *ctx, const srp_eval_params *prm)
{
    if (!prm) return fail(ctx, SRP_ERR_ARG, "null params");
    if (prm->N < 1 || prm->N > SRP_MAX_N) return fail(ctx, SRP_ERR_ARG, "N = %d outside [1, %d]", prm->N, SRP_MAX_N);
    if (prm->bounces < 0 || prm->bounces > kMaxBounces) return fail(ctx, SRP_ERR_ARG, "bounces = %d", prm->bounces);
    if (!(prm->P0 >= 0.0) || !(prm->eps_rel >= 0.0)) return fail(ctx, SRP_ERR_ARG, "P0 and eps_rel must be >= 0");
    if (prm->panel_mode < 0 || prm->panel_mode > 2) return fail(ctx, SRP_ERR_ARG, "bad panel_mode");
    if (prm->n_diffuse < 0 || prm->n_diffuse > SRP_MAX_DIFFUSE)
        return fail(ctx, SRP_ERR_ARG, "n_diffuse = %d outside [0, %d]", prm->n_diffuse, SRP_MAX_DIFFUSE);
    return SRP_OK;
}

// Launch shape of a batch of n evaluations.
struct EvalPlan {
    int N, nseg, S, nchunks, lanes, nbx, tw;
    size_t R, SL;
    int nba = 0, wa = 0;  // adjoint: ray blocks per slot, doubles per block partial
};

// Adjoint inputs of one batch (device pointers); null for a plain evaluation.
struct AdjBatch {
    const double *sun, *dist, *gF, *gT;
    double *g_sun, *g_dist, *g_eval;
    int panel_mode;
};

// Phase timing with CUDA events recorded on the stream each phase runs on.
struct Timing {
    srp_ctx *ctx;
    bool on;
    int n = 0;
    std::vector<std::pair<int, int>> spans[6];  // geometry, trace, refine, reduce, transfer, raster
    Timing(srp_ctx *c, bool o) : ctx(c), on(o) {}
    int mark(cudaStream_t s)
    {
        if (!on) return -1;
        if (n >= (int)ctx->events.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            ctx->events.push_back(e);
        }
        cudaEventRecord(ctx->events[n], s);
        return n++;
    }
    void span(int phase, int a, int b) { if (on) spans[phase].push_back({a, b}); }
    void collect(srp_eval_stats &L)
    {
        if (!on) return;
        double *ms[6] = {&L.ms_geometry, &L.ms_trace, &L.ms_refine, &L.ms_reduce, &L.ms_transfer, &L.ms_raster};
        for (int p = 0; p < 6; p++)
            for (auto &sp : spans[p]) {
                float t = 0.f;
                if (sp.first >= 0 && sp.second >= 0 &&
                    cudaEventElapsedTime(&t, ctx->events[sp.first], ctx->events[sp.second]) == cudaSuccess)
                    *ms[p] += t;
            }
    }
};

void fill_stats(srp_eval_stats &L, const unsigned long long *stats)
{
    L.evals = (int64_t)stats[0];
    L.rays = (int64_t)stats[1];
    L.refined = (int64_t)stats[2];
    L.segments = (int64_t)stats[3];
    for (int k = 0; k <= kMaxBounces; k++) L.hits[k] = (int64_t)stats[4 + k];
    L.nodes_visited = (int64_t)stats[9];
    L.tris_tested = (int64_t)stats[10];
    L.box_tests = (int64_t)stats[11];
    for (int k = 0; k < 4; k++) L.handoff_cause[k] = (int64_t)stats[12 + k];
}

// Trace tiles of a grid of N x N rays with tiles tw pixels wide (32 / tw high).
void tile_grid(int N, int tw, int &tiles_x, int &tiles)
{
    const int th = kTileRays / tw;
    tiles_x = (N + tw - 1) / tw;
    tiles = tiles_x * ((N + th - 1) / th);
}

// Slot k of the strided per-mesh slot buffers allocated by ensure_slots.
SlotBufs slot_bufs(const MeshDev &h, const SlotBufs &base, size_t k)
{
    SlotBufs b = base;
    b.vert64 += k * h.n_dyn_verts * 3;
    b.vview += k * h.n_verts;
    b.vview64 += k * h.n_verts * 3;
    b.tri += k * h.n_dyn_tris * 3;
    b.node += k * h.n_dyn_nodes * kNode4;
    b.counter += k * h.n_dyn_nodes;
    b.root_box += k * kMaxParts * 6;
    return b;
}

// Upload the slot descriptors unless the device already holds exactly these.
srp_status upload_slots(srp_ctx *ctx, const std::vector<SlotDesc> &sd)
{
    if (ctx->sdesc && ctx->sdesc_host.size() == sd.size() &&
        memcmp(ctx->sdesc_host.data(), sd.data(), sizeof(SlotDesc) * sd.size()) == 0)
        return SRP_OK;
    CK(ctx, grow(&ctx->sdesc, &ctx->sdesc_cap, sd.size(), false));
    CK(ctx, cudaMemcpy(ctx->sdesc, sd.data(), sizeof(SlotDesc) * sd.size(), cudaMemcpyHostToDevice));
    ctx->sdesc_host = sd;
    return SRP_OK;
}

int tuned_tile_w(const srp_ctx *ctx, const Mesh *m, int N, int nseg)
{
    auto it = ctx->tile_w.find(std::make_tuple((const void *)m, N, nseg));
    return it == ctx->tile_w.end() ? 8 : it->second;
}

// Size the batch and grow every buffer it needs (may allocate; never inside a capture).
srp_status eval_plan(srp_ctx *ctx, Mesh *m, const srp_eval_params *prm, int n, bool want_hits, EvalPlan &pl,
                     bool adjoint = false)
{
    pl.N = prm->N;
    pl.nseg = prm->bounces + 1;
    pl.R = (size_t)pl.N * pl.N;
    // concurrent evaluations: enough rays in flight to fill the GPU several times
    pl.S = (int)std::min<size_t>(std::max<size_t>((size_t)(1u << 23) / pl.R, 1), 32);
    pl.S = std::min(pl.S, std::max(n, 1));
    // chunks of S evaluations alternate between lane streams with their own
    // slots and buffers, so the short, latency-bound tail of one chunk (FP64
    // re-trace, reduction) overlaps the traversal of the next
    pl.nchunks = (n + pl.S - 1) / pl.S;
    pl.lanes = (prm->flags & SRP_EVAL_SERIAL) ? 1 : std::max(1, std::min(pl.nchunks, kLanes));
    srp_status rc = ensure_slots(ctx, m, pl.S * pl.lanes);
    if (rc) return rc;
    // trace tiles of 32 pixels, one warp each (shape from the autotuner, else 8 x 4)
    pl.tw = tuned_tile_w(ctx, m, pl.N, pl.nseg);
    int tiles_x = 0;
    tile_grid(pl.N, pl.tw, tiles_x, pl.nbx);
    pl.SL = (size_t)pl.S * pl.lanes;
    const size_t SL = pl.SL;
    CK(ctx, grow(&ctx->pose, &ctx->pose_cap, SL, false));
    CK(ctx, grow(&ctx->partials, &ctx->partials_cap, SL * pl.nbx * 6, false));
    CK(ctx, grow(&ctx->pcounts, &ctx->pcounts_cap, SL * pl.nbx * kCnt, false));
    CK(ctx, grow(&ctx->amb_list, &ctx->amb_list_cap, SL * pl.nbx * kTileRays, false));
    CK(ctx, grow(&ctx->partials1, &ctx->partials1_cap, SL * kRed1 * kPart, false));
    CK(ctx, grow(&ctx->red_ticket, &ctx->red_ticket_cap, SL, true));
    CK(ctx, grow(&ctx->tctx, &ctx->tctx_cap, SL * trace_ctx_bytes(), false));
    CK(ctx, grow(&ctx->amb_count, &ctx->amb_count_cap, SL * pl.nbx, false));
    if (!(prm->flags & SRP_EVAL_TRAVERSE)) {
        CK(ctx, grow(&ctx->pix_key, &ctx->pix_key_cap, SL * pl.R, false));
        CK(ctx, grow(&ctx->pix_cand, &ctx->pix_cand_cap, SL * pl.R * kPixCand, false));
        CK(ctx, grow(&ctx->big, &ctx->big_cap, (size_t)pl.lanes * pl.S * kBigPerSlot, false));
        CK(ctx, grow_fill(&ctx->big_count, &ctx->big_count_cap, (size_t)kLanes, 0));
        CK(ctx, grow(&ctx->bigt, &ctx->bigt_cap, (size_t)pl.lanes * pl.S * kBigPerSlot, false));
        CK(ctx, grow_fill(&ctx->bigt_count, &ctx->bigt_count_cap, (size_t)kLanes, 0));
        CK(ctx, grow_fill(&ctx->rast_bad, &ctx->rast_bad_cap, SL, 0));
        if (prm->flags & (SRP_EVAL_QUEUE | SRP_EVAL_TEST_WAIT_TIMEOUT))
            CK(ctx, grow(&ctx->qstate, &ctx->qstate_cap, (size_t)pl.lanes * qstate_words(pl.S), false));
    }
    // the diffuse rays replay each ray's recorded hits
    if (want_hits || adjoint || prm->n_diffuse > 0) CK(ctx, grow(&ctx->hits, &ctx->hits_cap, SL * pl.R * pl.nseg, false));
    if (prm->n_diffuse > 0) {
        CK(ctx, grow(&ctx->dpart, &ctx->dpart_cap, SL * kDiffBlocks * 6, false));
        if (pl.nseg > 1) {
            CK(ctx, grow(&ctx->demit, &ctx->demit_cap, SL * pl.R * (size_t)(pl.nseg - 1), false));
            CK(ctx, grow(&ctx->dcnt, &ctx->dcnt_cap, SL * pl.R, false));
            CK(ctx, grow(&ctx->dtot, &ctx->dtot_cap, SL, false));
        }
    }
    // every slot evaluates this mesh on this grid; lane b owns slots [b S, (b + 1) S)
    std::vector<SlotDesc> sd(SL);
    for (size_t k = 0; k < SL; k++) {
        SlotDesc &d = sd[k];
        d.mesh = m->d;
        d.sb = slot_bufs(m->h, m->sb, k);
        d.angles = m->angles_d;
        d.N = pl.N;
        d.nseg = pl.nseg;
        d.panel_mode = prm->panel_mode;
        d.tile_w = pl.tw;
        d.tiles_x = tiles_x;
        d.tiles = pl.nbx;
        d.tile0 = (int)(k % pl.S) * trace_blocks(pl.nbx);
        d.rast0 = (int)(k % pl.S) * ((m->h.n_tris + 127) / 128);
    }
    rc = upload_slots(ctx, sd);
    if (rc) return rc;
    if (adjoint) {
        pl.nba = adj_blocks(pl.S, pl.R);
        pl.wa = kAdjFixed + 2 * m->h.n_mats + 6 * m->h.n_parts;
        CK(ctx, grow(&ctx->adj_partials, &ctx->adj_partials_cap, SL * pl.nba * pl.wa, false));
        CK(ctx, grow(&ctx->adj_partials2, &ctx->adj_partials2_cap,
                     SL * (size_t)((pl.nba + kAdjSumRun - 1) / kAdjSumRun) * pl.wa, false));
        CK(ctx, grow(&ctx->win_ids, &ctx->win_ids_cap, SL * 4, false));
        CK(ctx, grow(&ctx->win_val, &ctx->win_val_cap, SL * kAdjWinBlocks * 4, false));
        CK(ctx, grow(&ctx->win_pid, &ctx->win_pid_cap, SL * kAdjWinBlocks * 4, false));
    }
    return SRP_OK;
}

// Queue the evaluations on the lane streams, forked from and joined back into
// the context stream.  Launches and event records only: no allocation, no
// synchronisation, so a stream capture can record it.
srp_status eval_enqueue(srp_ctx *ctx, Mesh *m, const srp_eval_params *prm, const EvalPlan &pl, int n,
                        const double *d_sun, const double *d_dist, double *d_f, double *d_t, int32_t *hit_tri,
                        bool h_dev, Timing &tm, int64_t &launches, int64_t &trace_launches,
                        const AdjBatch *adj = nullptr)
{
    cudaStream_t st = ctx->stream;
    const int S = pl.S, nbx = pl.nbx, nseg = pl.nseg;
    const size_t R = pl.R;
    const int h_tris = m->h.n_tris;
    CK(ctx, cudaEventRecord(ctx->ev_fork, st));
    for (int b = 0; b < pl.lanes; b++) CK(ctx, cudaStreamWaitEvent(ctx->lane[b], ctx->ev_fork, 0));
    for (int c = 0; c < pl.nchunks; c++) {
        const int e0 = c * S, b = c % pl.lanes;
        const int Sc = std::min(S, n - e0);
        cudaStream_t ls = ctx->lane[b];
        // lane b's slots and buffers
        const MeshDev &h = m->h;
        size_t s0 = (size_t)b * S;
        const SlotDesc *sd = ctx->sdesc + s0;
        SlotPose *pose = ctx->pose + s0;
        TraceArgs a{};
        a.sd = sd;
        a.n_slots = Sc;
        a.n_tiles = Sc * trace_blocks(nbx);
        a.pose = pose;
        a.ray_stride = R;
        a.seg_stride = nseg;
        a.eps_rel = prm->eps_rel;
        a.n_blocks_x = nbx;
        a.partials = ctx->partials + s0 * nbx * 6;
        a.pcounts = ctx->pcounts + s0 * nbx * kCnt;
        a.partials1 = ctx->partials1 + s0 * kRed1 * kPart;
        a.red_ticket = ctx->red_ticket + s0;
        a.tctx = ctx->tctx + s0 * trace_ctx_bytes();
        a.amb_list = ctx->amb_list + s0 * nbx * kTileRays;
        a.amb_count = ctx->amb_count + s0 * nbx;
        a.count = (prm->flags & SRP_EVAL_COUNT) ? 1 : 0;
        if (!(prm->flags & SRP_EVAL_TRAVERSE)) {
            a.raster = 1;
            a.rast_tris = h_tris;
            a.pix_key = ctx->pix_key + s0 * R;
            a.pix_cand = ctx->pix_cand + s0 * R * kPixCand;
            a.big_cap = S * kBigPerSlot;
            a.big = ctx->big + (size_t)b * a.big_cap;
            a.big_count = ctx->big_count + b;
            a.bigt = ctx->bigt + (size_t)b * a.big_cap;
            a.bigt_count = ctx->bigt_count + b;
            a.rast_bad = ctx->rast_bad + s0;
            if (prm->flags & (SRP_EVAL_QUEUE | SRP_EVAL_TEST_WAIT_TIMEOUT)) {
                a.queue = 1;
                a.wait_test = (prm->flags & SRP_EVAL_TEST_WAIT_TIMEOUT) ? 1 : 0;
                a.n_small_items = Sc * ((h_tris + 127) / 128);
                a.qstate = ctx->qstate + (size_t)b * qstate_words(S);
            }
        }
        int32_t *stage = ctx->hits ? ctx->hits + s0 * R * nseg : nullptr;
        a.hits = hit_tri ? (h_dev ? hit_tri + (size_t)e0 * R * nseg : stage) : ((adj || prm->n_diffuse > 0) ? stage : nullptr);
        a.walk_limit_test = (prm->flags & SRP_EVAL_TEST_WALK_BOUND) ? 1 : 0;
        a.sum_mode = (prm->flags & SRP_EVAL_SUM_COMP32) ? 1 : ((prm->flags & SRP_EVAL_SUM_FP32) ? 2 : 0);
        a.ctx_parts = h.n_parts;
        a.hpt_segs = nseg;
        if (prm->n_diffuse > 0 && nseg > 1) {
            a.n_diffuse = prm->n_diffuse;
            a.diffuse_seed = prm->diffuse_seed;
            a.dpart = ctx->dpart + s0 * kDiffBlocks * 6;
            a.demit = ctx->demit + s0 * R * (size_t)(nseg - 1);
            a.dcnt = ctx->dcnt + s0 * R;
            a.dtot = ctx->dtot + s0;
        }
        int g0 = tm.mark(ls);
        CK(ctx, launch_pose(sd, d_sun, d_dist, prm->P0, e0, Sc, pose, ls));
        CK(ctx, launch_vertices(sd, pose, Sc, h.n_verts, ls));
        launches += 2;
        // the refit feeds only the trace (the raster reads the posed view-frame
        // vertices): it runs on the lane's side stream beside frame and raster
        const bool refit = h.n_dyn_tris > 0;
        if (refit) {
            CK(ctx, cudaEventRecord(ctx->ev_refit_fork[b], ls));
            CK(ctx, cudaStreamWaitEvent(ctx->aux[b], ctx->ev_refit_fork[b], 0));
            CK(ctx, launch_refit(sd, pose, Sc, h.n_dyn_tris, ctx->aux[b]));
            CK(ctx, cudaEventRecord(ctx->ev_refit_join[b], ctx->aux[b]));
            launches++;
        }
        int g1 = tm.mark(ls);
        CK(ctx, launch_frame(a, Sc, ls));
        if (refit) CK(ctx, cudaStreamWaitEvent(ls, ctx->ev_refit_join[b], 0));
        int g1r = tm.mark(ls);
        CK(ctx, launch_trace(a, Sc, ls));
        int g2 = tm.mark(ls);
        int g3 = g2;  // the FP64 re-trace of overflowing rays runs inside the first reduction level
        CK(ctx, launch_reduce(a, Sc, e0, d_f, d_t, ctx->err_flags, ctx->stats, ls));
        int g4 = tm.mark(ls);
        launches += a.n_diffuse > 0 ? 4 : 3;  // frame, trace, the reduction (two levels in one launch without diffuse rays)
        if (a.raster) launches += raster_launches(Sc, a.queue != 0);
        if (a.n_diffuse > 0) launches += 3;  // diffuse secondaries: emission records, their prefix, the rays
        trace_launches++;
        if (adj) {
            AdjArgs g{};
            g.sd = sd;
            g.pose = pose;
            g.hits = a.hits;
            g.ray_stride = R;
            g.seg_stride = nseg;
            g.sun_dirs = adj->sun;
            g.sun_dist = adj->dist;
            g.g_force = adj->gF;
            g.g_torque = adj->gT;
            g.panel_mode = adj->panel_mode;
            g.n_mats = h.n_mats;
            g.n_parts = h.n_parts;
            g.eval0 = e0;
            g.nb = pl.nba;
            g.width = pl.wa;
            g.win_ids = ctx->win_ids + s0 * 4;
            g.win_val = ctx->win_val + s0 * kAdjWinBlocks * 4;
            g.win_pid = ctx->win_pid + s0 * kAdjWinBlocks * 4;
            g.n_verts = h.n_verts;
            g.partials = ctx->adj_partials + s0 * pl.nba * pl.wa;
            g.partials2 = ctx->adj_partials2 + s0 * (size_t)((pl.nba + kAdjSumRun - 1) / kAdjSumRun) * pl.wa;
            g.g_sun = adj->g_sun;
            g.g_dist = adj->g_dist;
            g.g_eval = adj->g_eval;
            CK(ctx, launch_adjoint(g, Sc, ls));
            launches += 4;  // window search and merge, rays, finish
        }
        tm.span(0, g0, g1);
        tm.span(5, g1, g1r);
        tm.span(1, g1r, g2);
        tm.span(2, g2, g3);
        tm.span(3, g3, g4);
        if (hit_tri && !h_dev) {
            CK(ctx, cudaMemcpyAsync(hit_tri + (size_t)e0 * R * nseg, stage, sizeof(int32_t) * Sc * R * nseg,
                                    cudaMemcpyDeviceToHost, ls));
            tm.span(4, g4, tm.mark(ls));
        }
    }
    // join: the context stream continues after every lane
    for (int b = 0; b < pl.lanes; b++) {
        CK(ctx, cudaEventRecord(ctx->ev_join[b], ctx->lane[b]));
        CK(ctx, cudaStreamWaitEvent(st, ctx->ev_join[b], 0));
    }
    return SRP_OK;
}

// Adjoint of evaluations whose hits were recorded earlier: posing and window
// vertices again (no trace), then the frozen-hit reverse sweep, on `st` with
// the first lane's slots.  hits: [n][N*N][nseg] original triangle ids.
srp_status adj_enqueue(srp_ctx *ctx, Mesh *m, const srp_eval_params *prm, const EvalPlan &pl, int n,
                       const double *d_sun, const double *d_dist, const int32_t *hits, const AdjBatch &ab,
                       cudaStream_t st, int64_t &launches)
{
    const MeshDev &h = m->h;
    for (int e0 = 0; e0 < n; e0 += pl.S) {
        const int Sc = std::min(pl.S, n - e0);
        SlotPose *pose = ctx->pose;
        const SlotDesc *sd = ctx->sdesc;
        CK(ctx, launch_pose(sd, d_sun, d_dist, prm->P0, e0, Sc, pose, st));
        CK(ctx, launch_vertices(sd, pose, Sc, h.n_verts, st));
        AdjArgs g{};
        g.sd = sd;
        g.pose = pose;
        g.hits = hits + (size_t)e0 * pl.R * pl.nseg;
        g.ray_stride = pl.R;
        g.seg_stride = pl.nseg;
        g.sun_dirs = d_sun;
        g.sun_dist = ab.dist;
        g.g_force = ab.gF;
        g.g_torque = ab.gT;
        g.panel_mode = ab.panel_mode;
        g.n_mats = h.n_mats;
        g.n_parts = h.n_parts;
        g.eval0 = e0;
        g.nb = pl.nba;
        g.width = pl.wa;
        g.win_ids = ctx->win_ids;
        g.win_val = ctx->win_val;
        g.win_pid = ctx->win_pid;
        g.n_verts = h.n_verts;
        g.partials = ctx->adj_partials;
        g.partials2 = ctx->adj_partials2;
        g.g_sun = ab.g_sun;
        g.g_dist = ab.g_dist;
        g.g_eval = ab.g_eval;
        CK(ctx, launch_adjoint(g, Sc, st));
        launches += 6;  // pose, vertices, window search and merge, rays, finish
    }
    return SRP_OK;
}

PropDev prop_dev(const srp_prop_params *p, const Mesh *m)
{
    PropDev P{};
    P.method = p->method; P.central = p->central; P.j2 = p->j2; P.sun3 = p->sun3; P.srp = p->srp;
    P.attitude = p->attitude;
    for (int k = 0; k < 4; k++) P.q[k] = p->q[k];
    P.epoch_mjd_tt = p->epoch_mjd_tt; P.mass = m->mass;
    P.rtol = p->rtol; P.atol_pos = p->atol_pos; P.atol_vel = p->atol_vel;
    P.h0 = p->h0; P.h_min = p->h_min; P.h_max = p->h_max; P.max_steps = p->max_steps;
    return P;
}

// Number of fixed RK4 steps from t0 to t1 (the last one shortened to land on
// t1, a step ending within 1e-9 h0 of t1 snapped onto it), as k_prop_control
// takes them; -1 beyond max_steps.
int64_t rk4_steps(double t0, double t1, double h0, int64_t max_steps)
{
    int64_t k = 0;
    double t = t0;
    while (t < t1) {
        const bool last = t + h0 >= t1;
        const double h = last ? t1 - t : h0;
        t = (last || t1 - (t + h) < 1e-9 * h0) ? t1 : t + h;
        if (++k > max_steps) return -1;
    }
    return k;
}

// Read back the trajectories: final states, per-trajectory stats, step log.
srp_status finish_propagate(srp_ctx *ctx, int n, const PropState *S, double *y1, srp_prop_stats *stats, double *h_log,
                            int64_t h_cap)
{
    cudaStream_t st = ctx->stream;
    std::vector<PropState> hs(n);
    int flags = 0;
    unsigned long long st16[16];
    CK(ctx, cudaMemcpyAsync(hs.data(), S, sizeof(PropState) * n, cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaMemcpyAsync(&flags, ctx->err_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaMemcpyAsync(st16, ctx->stats, sizeof st16, cudaMemcpyDeviceToHost, st));
    if (h_log) CK(ctx, cudaMemcpyAsync(h_log, ctx->prop_hlog, sizeof(double) * n * h_cap, cudaMemcpyDefault, st));
    CK(ctx, cudaStreamSynchronize(st));
    std::vector<double> yo((size_t)n * 6);
    srp_status out = SRP_OK;
    for (int i = 0; i < n; i++) {
        for (int k = 0; k < 6; k++) yo[6 * (size_t)i + k] = hs[i].y[k];
        if (stats) {
            stats[i].steps = hs[i].steps;
            stats[i].rejects = hs[i].rejects;
            stats[i].evals = hs[i].evals;
            stats[i].t = hs[i].t;
            stats[i].status = hs[i].status;
            stats[i].reserved = 0;
            stats[i].h_next = hs[i].h;
        }
        if (hs[i].status) out = SRP_ERR_STEP;
        if (!hs[i].done) out = fail(ctx, SRP_ERR_STEP, "trajectory %d did not finish within the step budget", i);
    }
    CK(ctx, cudaMemcpy(y1, yo.data(), sizeof(double) * 6 * n, cudaMemcpyDefault));
    fill_stats(ctx->last, st16);
    if (flags & kFlagTimeout) return fail(ctx, SRP_ERR_TIMEOUT, "a work-queue wait gave up");
    if (flags & kFlagStack) return fail(ctx, SRP_ERR_STACK, "traversal stack bound reached");
    if (out == SRP_ERR_STEP && ctx->err.empty()) fail(ctx, SRP_ERR_STEP, "a trajectory hit h_min or max_steps");
    return out;
}

}  // namespace

// ======================================================================= ABI
srp_status check_spad_grid(srp_ctx *ctx, const srp_spad_grid *g)
{
    if (!g) return fail(ctx, SRP_ERR_ARG, "null SPAD grid");
    if (g->n_az < 1 || g->n_el < 1 || g->n_az > (1 << 20) || g->n_el > (1 << 20) ||
        (int64_t)g->n_az * g->n_el > (int64_t)1 << 24)
        return fail(ctx, SRP_ERR_ARG, "SPAD grid needs 1 <= n_az, n_el <= 2^20 and n_az n_el <= 2^24");
    if (!std::isfinite(g->az0) || !std::isfinite(g->el0) || !std::isfinite(g->d_el) || !(g->d_el > 0.0))
        return fail(ctx, SRP_ERR_ARG, "SPAD grid needs finite az0, el0 and d_el > 0");
    return SRP_OK;
}

SpadDev spad_dev(const srp_spad_grid *g, const double *table)
{
    SpadDev d{};
    d.table = table;
    d.n_az = g->n_az;
    d.n_el = g->n_el;
    d.az0 = g->az0;
    d.el0 = g->el0;
    d.d_el = g->d_el;
    return d;
}

extern "C" {

srp_status srp_create(srp_ctx **out, int32_t device, void *cuda_stream)
{
    if (!out) return SRP_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return SRP_ERR_CUDA;
    }
    srp_ctx *ctx = new (std::nothrow) srp_ctx();
    if (!ctx) return SRP_ERR_OOM;
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess) { delete ctx; return SRP_ERR_CUDA; }
    if (configure_trace_kernels() != cudaSuccess) { cudaGetLastError(); delete ctx; return SRP_ERR_CUDA; }
    if (cuda_stream) {
        ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return SRP_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    if (dalloc(&ctx->err_flags, sizeof(int)) != cudaSuccess ||
        dalloc(&ctx->stats, 16 * sizeof(unsigned long long)) != cudaSuccess ||
        dalloc(&ctx->prop_done, sizeof(int)) != cudaSuccess) {
        srp_destroy(ctx);
        return SRP_ERR_OOM;
    }
    for (int b = 0; b < kLanes; b++)
        if (cudaStreamCreateWithFlags(&ctx->lane[b], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_join[b], cudaEventDisableTiming) != cudaSuccess ||
            cudaStreamCreateWithFlags(&ctx->aux[b], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_refit_fork[b], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_refit_join[b], cudaEventDisableTiming) != cudaSuccess) {
            srp_destroy(ctx);
            return SRP_ERR_CUDA;
        }
    if (cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
        srp_destroy(ctx);
        return SRP_ERR_CUDA;
    }
    *out = ctx;
    return SRP_OK;
}

void srp_destroy(srp_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (Mesh *m : ctx->meshes) free_mesh(m);
    dfree(ctx->pose);
    dfree(ctx->partials);
    dfree(ctx->pcounts);
    dfree(ctx->amb_list);
    dfree(ctx->partials1);
    dfree(ctx->red_ticket);
    dfree(ctx->dpart);
    dfree(ctx->demit);
    dfree(ctx->dcnt);
    dfree(ctx->dtot);
    dfree(ctx->tctx);
    dfree(ctx->prop_io);
    dfree(ctx->spad_buf);
    dfree(ctx->prop_state);
    dfree(ctx->prop_hlog);
    dfree(ctx->prop_replay);
    dfree(ctx->prop_done);
    dfree(ctx->amb_count);
    dfree(ctx->pix_key);
    dfree(ctx->qstate);
    dfree(ctx->pix_cand);
    dfree(ctx->big);
    dfree(ctx->big_count);
    dfree(ctx->bigt);
    dfree(ctx->bigt_count);
    dfree(ctx->rast_bad);
    dfree(ctx->io);
    dfree(ctx->hits);
    dfree(ctx->adj_partials);
    dfree(ctx->adj_partials2);
    dfree(ctx->win_ids);
    dfree(ctx->win_val);
    dfree(ctx->win_pid);
    dfree(ctx->gio);
    dfree(ctx->sdesc);
    dfree(ctx->arc_hits);
    dfree(ctx->arc_buf);
    dfree(ctx->err_flags);
    dfree(ctx->stats);
    for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
    for (int b = 0; b < kLanes; b++) {
        if (ctx->lane[b]) cudaStreamSynchronize(ctx->lane[b]), cudaStreamDestroy(ctx->lane[b]);
        if (ctx->ev_join[b]) cudaEventDestroy(ctx->ev_join[b]);
        if (ctx->aux[b]) cudaStreamSynchronize(ctx->aux[b]), cudaStreamDestroy(ctx->aux[b]);
        if (ctx->ev_refit_fork[b]) cudaEventDestroy(ctx->ev_refit_fork[b]);
        if (ctx->ev_refit_join[b]) cudaEventDestroy(ctx->ev_refit_join[b]);
    }
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char *srp_last_error(const srp_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

srp_status srp_mesh_load(srp_ctx *ctx, const srp_mesh_desc *D, int32_t *mesh_id)
{
    if (!ctx) return SRP_ERR_ARG;
    ctx->err.clear();
    if (!D || !mesh_id) return fail(ctx, SRP_ERR_ARG, "null desc or mesh_id");
    if (D->n_verts <= 0 || D->n_tris <= 0 || D->n_parts <= 0 || D->n_mats <= 0)
        return fail(ctx, SRP_ERR_ARG, "counts must be positive");
    if (D->n_parts > kMaxParts) return fail(ctx, SRP_ERR_ARG, "n_parts %d > %d", D->n_parts, kMaxParts);
    if (D->n_mats > kMaxMats) return fail(ctx, SRP_ERR_ARG, "n_mats %d > %d", D->n_mats, kMaxMats);
    if (!D->xyz || !D->tri || !D->tri_part || !D->tri_mat || !D->mat || !D->parent || !D->pivot || !D->axis ||
        !D->limits || !D->normal0)
        return fail(ctx, SRP_ERR_ARG, "null array in mesh description");
    if (D->vertex_dtype != SRP_F32 && D->vertex_dtype != SRP_F64) return fail(ctx, SRP_ERR_ARG, "bad vertex dtype");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, SRP_ERR_CUDA, "cudaSetDevice");
    const int NV = D->n_verts, NT = D->n_tris, NP = D->n_parts, NM = D->n_mats;
    // ---- validation
    std::vector<double> xyz((size_t)NV * 3);
    for (size_t k = 0; k < xyz.size(); k++) {
        xyz[k] = D->vertex_dtype == SRP_F64 ? static_cast<const double *>(D->xyz)[k]
                                            : (double)static_cast<const float *>(D->xyz)[k];
        if (!std::isfinite(xyz[k])) return fail(ctx, SRP_ERR_MESH, "non-finite vertex coordinate %zu", k / 3);
    }
    if (D->parent[0] != -1) return fail(ctx, SRP_ERR_MESH, "parent[0] must be -1");
    std::vector<int> movable(NP, 0), dynamic(NP, 0);
    for (int p = 0; p < NP; p++) {
        if (p > 0 && (D->parent[p] < 0 || D->parent[p] >= p))
            return fail(ctx, SRP_ERR_MESH, "parent[%d] = %d must lie in [0, %d)", p, D->parent[p], p);
        const double *a = D->axis + 3 * p;
        double an = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        if (p > 0 && an != 0.0) {
            if (std::fabs(an - 1.0) > 1e-9) return fail(ctx, SRP_ERR_MESH, "axis of part %d is not unit", p);
            movable[p] = 1;
        }
        if (!(D->limits[2 * p] <= D->limits[2 * p + 1])) return fail(ctx, SRP_ERR_MESH, "limits of part %d", p);
        dynamic[p] = movable[p] || (p > 0 && dynamic[D->parent[p]]);
    }
    for (int i = 0; i < NM; i++) {
        double rs = D->mat[2 * i], rd = D->mat[2 * i + 1];
        if (!(rs >= 0.0 && rd >= 0.0 && rs + rd <= 1.0 + 1e-12))
            return fail(ctx, SRP_ERR_MESH, "material %d coefficients (%g, %g) outside [0,1] or sum > 1", i, rs, rd);
    }
    std::vector<int> vpart(NV, -1);
    for (int t = 0; t < NT; t++) {
        int p = D->tri_part[t];
        if (p < 0 || p >= NP) return fail(ctx, SRP_ERR_MESH, "tri_part[%d] = %d out of range", t, p);
        for (int s = 0; s < 2; s++)
            if (D->tri_mat[2 * t + s] < 0 || D->tri_mat[2 * t + s] >= NM)
                return fail(ctx, SRP_ERR_MESH, "tri_mat[%d] out of range", t);
        for (int c = 0; c < 3; c++) {
            int v = D->tri[3 * t + c];
            if (v < 0 || v >= NV) return fail(ctx, SRP_ERR_MESH, "tri[%d] vertex %d out of range", t, v);
            if (vpart[v] >= 0 && vpart[v] != p) return fail(ctx, SRP_ERR_MESH, "vertex %d shared by parts %d and %d", v, vpart[v], p);
            vpart[v] = p;
        }
        const double *a = &xyz[3 * (size_t)D->tri[3 * t]], *b = &xyz[3 * (size_t)D->tri[3 * t + 1]],
                     *c = &xyz[3 * (size_t)D->tri[3 * t + 2]];
        double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        if (!(n[0] * n[0] + n[1] * n[1] + n[2] * n[2] > 0.0)) return fail(ctx, SRP_ERR_MESH, "triangle %d is degenerate", t);
    }
    {
        // a hit is recorded as (part << 24) | the triangle's index within its part
        std::vector<int> per_part(NP, 0);
        for (int t = 0; t < NT; t++) per_part[D->tri_part[t]]++;
        for (int p = 0; p < NP; p++)
            if (per_part[p] >= (1 << 24))
                return fail(ctx, SRP_ERR_MESH, "part %d has %d triangles (at most %d a part)", p, per_part[p], (1 << 24) - 1);
    }
    // ---- layout: static parts first, then dynamic; vertices and triangles grouped by part
    std::vector<int> order;
    for (int p = 0; p < NP; p++) if (!dynamic[p]) order.push_back(p);
    for (int p = 0; p < NP; p++) if (dynamic[p]) order.push_back(p);
    std::vector<int> rank(NP);
    for (int r = 0; r < NP; r++) rank[order[r]] = r;
    std::vector<std::vector<int>> pverts(NP), ptris(NP);
    for (int v = 0; v < NV; v++) if (vpart[v] >= 0) pverts[vpart[v]].push_back(v);
    for (int t = 0; t < NT; t++) ptris[D->tri_part[t]].push_back(t);
    Mesh *m = new (std::nothrow) Mesh();
    if (!m) return fail(ctx, SRP_ERR_OOM, "host allocation");
    MeshDev &h = m->h;
    h.n_parts = NP; h.n_tris = NT; h.n_mats = NM;
    std::vector<int> newv(NV, -1);
    std::vector<double> rest;
    std::vector<int> vert_part;
    int nv = 0, tb = 0, nb = 0;
    std::vector<int> bin_begin(NP, 0);
    double rmax = 0.0, piv = 0.0;
    for (int r = 0; r < NP; r++) {
        int p = order[r];
        PartInfo &pi = h.part[p];
        pi.parent = D->parent[p];
        pi.movable = movable[p];
        pi.dynamic = dynamic[p];
        for (int k = 0; k < 3; k++) {
            pi.pivot[k] = D->pivot[3 * p + k];
            pi.axis[k] = D->axis[3 * p + k];
            pi.n0[k] = D->normal0[3 * p + k];
        }
        pi.lim[0] = D->limits[2 * p];
        pi.lim[1] = D->limits[2 * p + 1];
        pi.vert_begin = nv;
        pi.vert_count = (int)pverts[p].size();
        for (int v : pverts[p]) {
            newv[v] = nv++;
            for (int k = 0; k < 3; k++) rest.push_back(xyz[3 * (size_t)v + k]);
            vert_part.push_back(p);
            rmax = std::max(rmax, std::sqrt(xyz[3 * (size_t)v] * xyz[3 * (size_t)v] +
                                            xyz[3 * (size_t)v + 1] * xyz[3 * (size_t)v + 1] +
                                            xyz[3 * (size_t)v + 2] * xyz[3 * (size_t)v + 2]));
        }
        pi.tri_begin = tb;
        pi.tri_count = (int)ptris[p].size();
        tb += pi.tri_count;
        bin_begin[p] = nb;  // binary radix tree nodes of the part (collapsed to 4-wide after the build)
        nb += std::max(pi.tri_count - 1, 0);
        if (movable[p]) piv += std::sqrt(pi.pivot[0] * pi.pivot[0] + pi.pivot[1] * pi.pivot[1] + pi.pivot[2] * pi.pivot[2]);
        if (!dynamic[p]) { h.n_static_tris = tb; h.n_static_verts = nv; }
    }
    h.n_verts = nv;
    h.n_dyn_tris = NT - h.n_static_tris;
    h.n_dyn_verts = nv - h.n_static_verts;
    for (int p = 0; p < NP; p++) {
        PartInfo &pi = h.part[p];
        pi.dyn_tri_off = pi.dynamic ? pi.tri_begin - h.n_static_tris : 0;
        pi.dyn_vert_off = pi.dynamic ? pi.vert_begin - h.n_static_verts : 0;
        h.part_order[rank[p]] = p;
    }
    h.R = rmax + 2.0 * piv;
    h.pad = std::ldexp(h.R, -16) + 1e-9;
    for (int k = 0; k < 3; k++) h.c_ref[k] = D->c_ref[k];
    m->mass = D->mass;
    // part boxes for Morton quantisation
    std::vector<float> plo((size_t)NP * 3, 0.f), pext((size_t)NP * 3, 0.f);
    for (int p = 0; p < NP; p++) {
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int v : pverts[p])
            for (int k = 0; k < 3; k++) { lo[k] = std::min(lo[k], xyz[3 * (size_t)v + k]); hi[k] = std::max(hi[k], xyz[3 * (size_t)v + k]); }
        for (int k = 0; k < 3; k++) {
            plo[3 * p + k] = pverts[p].empty() ? 0.f : (float)lo[k];
            pext[3 * p + k] = pverts[p].empty() ? 0.f : (float)(hi[k] - lo[k]);
        }
    }
    std::vector<int> tvidx((size_t)NT * 3);
    for (int t = 0; t < NT; t++)
        for (int c = 0; c < 3; c++) tvidx[3 * (size_t)t + c] = newv[D->tri[3 * t + c]];
    std::vector<int> rank_v(rank.begin(), rank.end());
    std::vector<int> tpart(D->tri_part, D->tri_part + NT);
    std::vector<int> tgrp(NT, 0);
    std::vector<double> tdev(NT, 0.0);
    for (int p = 0; p < NP; p++) {
        double ext = std::max(std::max(pext[3 * p], pext[3 * p + 1]), pext[3 * p + 2]);
        coplanar_groups(ptris[p], D->tri, xyz, ext, tgrp, tdev);
    }

    cudaStream_t st = ctx->stream;
    std::vector<void *> tmp;  // build-only device buffers
    auto free_tmp = [&]() { cudaStreamSynchronize(st); for (void *p : tmp) dfree(p); tmp.clear(); };
    auto bail = [&](srp_status c, const char *what, cudaError_t e) {
        free_tmp();
        free_mesh(m);
        return fail(ctx, c, "%s: %s", what, cudaGetErrorString(e));
    };
#define MK(x)                                                                                               \
    do {                                                                                                    \
        cudaError_t e_ = (x);                                                                               \
        if (e_ != cudaSuccess) return bail(e_ == cudaErrorMemoryAllocation ? SRP_ERR_OOM : SRP_ERR_CUDA, #x, e_); \
    } while (0)
    int *d_tvidx0, *d_tpart, *d_tgrp, *d_rank, *vals, *vals2, *scratch, *d_ptb, *d_ptc, *d_pnb, *d_nodepart, *d_nodebase, *d_depth;
    unsigned long long *keys, *keys2;
    float *d_plo, *d_pext;
    int4 *node_refs;
    unsigned *cnt_static;
    size_t sc_ints = radix_sort_scratch_ints(NT);
    MK(dmalloc(m->allocs, &h.rest64, (size_t)nv * 3));
    MK(dmalloc(m->allocs, &h.vert_part, (size_t)nv));
    MK(dmalloc(m->allocs, &h.tri_vidx, (size_t)NT * 3));
    MK(dmalloc(m->allocs, &h.tri_v4, (size_t)NT));
    MK(dmalloc(m->allocs, &h.tri_orig, (size_t)NT));
    MK(dmalloc(m->allocs, &h.tri_pos, (size_t)NT));
    MK(dmalloc(m->allocs, &h.tri_mat, (size_t)NT));
    MK(dmalloc(m->allocs, &h.leaf_parent, (size_t)NT));
    MK(dmalloc(m->allocs, &h.tri_static, (size_t)std::max(h.n_static_tris, 1) * 3));
    MK(dmalloc(m->allocs, &h.mat32, (size_t)NM));
    MK(dmalloc(m->allocs, &h.mat64, (size_t)NM * 2));
    MK(dmalloc(m->allocs, &m->angles_d, (size_t)NP));
    MK(dmalloc(tmp, &node_refs, (size_t)std::max(nb, 1)));
    MK(dmalloc(tmp, &d_tvidx0, (size_t)NT * 3));
    MK(dmalloc(tmp, &d_tpart, (size_t)NT));
    MK(dmalloc(tmp, &d_tgrp, (size_t)NT));
    MK(dmalloc(m->allocs, &h.grp, (size_t)NT));
    MK(dmalloc(tmp, &d_rank, (size_t)NP));
    MK(dmalloc(tmp, &keys, (size_t)NT));
    MK(dmalloc(tmp, &keys2, (size_t)NT));
    MK(dmalloc(tmp, &vals, (size_t)NT));
    MK(dmalloc(tmp, &vals2, (size_t)NT));
    MK(dmalloc(tmp, &scratch, sc_ints));
    MK(dmalloc(tmp, &d_plo, (size_t)NP * 3));
    MK(dmalloc(tmp, &d_pext, (size_t)NP * 3));
    MK(dmalloc(tmp, &d_ptb, (size_t)NP));
    MK(dmalloc(tmp, &d_ptc, (size_t)NP));
    MK(dmalloc(tmp, &d_pnb, (size_t)NP));
    MK(dmalloc(tmp, &d_nodepart, (size_t)std::max(nb, 1)));
    MK(dmalloc(tmp, &d_nodebase, (size_t)std::max(nb, 1)));
    MK(dmalloc(tmp, &d_depth, 1));
    MK(cudaMemcpyAsync(h.rest64, rest.data(), sizeof(double) * rest.size(), cudaMemcpyHostToDevice, st));
    MK(cudaMemcpyAsync(h.vert_part, vert_part.data(), sizeof(int) * nv, cudaMemcpyHostToDevice, st));
    MK(cudaMemcpyAsync(d_tvidx0, tvidx.data(), sizeof(int) * tvidx.size(), cudaMemcpyHostToDevice, st));
    MK(cudaMemcpyAsync(d_tpart, tpart.data(), sizeof(int) * NT, cudaMemcpyHostToDevice, st));
    MK(cudaMemcpyAsync(d_tgrp, tgrp.data(), sizeof(int) * NT, cudaMemcpyHostToDevice, st));
    MK(cudaMemcpyAsync(d_rank, rank_v.data(), sizeof(int) * NP, cudaMemcpyHostToDevice, st));
    MK(cudaMemcpyAsync(d_plo, plo.data(), sizeof(float) * plo.size(), cudaMemcpyHostToDevice, st));
    MK(cudaMemcpyAsync(d_pext, pext.data(), sizeof(float) * pext.size(), cudaMemcpyHostToDevice, st));
    // 1-2: Morton codes and sort (bits 0..51 hold the code, the coplanar group and the part rank)
    MK(launch_morton(h.rest64, d_tvidx0, d_tpart, d_rank, d_tgrp, d_plo, d_pext, NT, keys, vals, st));
    MK(radix_sort_pairs(keys, vals, keys2, vals2, NT, 0, 56, scratch, sc_ints, st));
    std::vector<int> sorted(NT);
    MK(cudaMemcpyAsync(sorted.data(), vals, sizeof(int) * NT, cudaMemcpyDeviceToHost, st));
    MK(cudaStreamSynchronize(st));
    // sorted triangle arrays (a check that the sort kept parts contiguous comes for free)
    std::vector<int> svidx((size_t)NT * 3), sorig(NT);
    std::vector<unsigned> smat(NT);
    for (int k = 0; k < NT; k++) {
        int t = sorted[k];
        if (t < 0 || t >= NT) return bail(SRP_ERR_CUDA, "sort produced an invalid index", cudaErrorUnknown);
        sorig[k] = t;
        for (int c = 0; c < 3; c++) svidx[3 * (size_t)k + c] = tvidx[3 * (size_t)t + c];
        smat[k] = (unsigned)D->tri_mat[2 * t] | ((unsigned)D->tri_mat[2 * t + 1] << 16);
    }
    for (int r = 0; r < NP; r++) {
        const PartInfo &pi = h.part[order[r]];
        for (int k = pi.tri_begin; k < pi.tri_begin + pi.tri_count; k++)
            if (D->tri_part[sorig[k]] != order[r]) return bail(SRP_ERR_CUDA, "sort mixed parts", cudaErrorUnknown);
    }
    MK(cudaMemcpyAsync(h.tri_vidx, svidx.data(), sizeof(int) * svidx.size(), cudaMemcpyHostToDevice, st));
    // vertex ids, and in the fourth word the triangle's hit record (part << 24) |
    // index within the part, which the raster writes into the pixel keys
    std::vector<int4> sv4(NT);
    for (int k = 0; k < NT; k++) sv4[k] = make_int4(svidx[3 * (size_t)k], svidx[3 * (size_t)k + 1], svidx[3 * (size_t)k + 2], 0);
    for (int r = 0; r < NP; r++) {
        const int p = order[r];
        const PartInfo &pi = h.part[p];
        for (int k = pi.tri_begin; k < pi.tri_begin + pi.tri_count; k++) sv4[k].w = (p << 24) | (k - pi.tri_begin);
    }
    MK(cudaMemcpyAsync(h.tri_v4, sv4.data(), sizeof(int4) * NT, cudaMemcpyHostToDevice, st));
    MK(cudaMemcpyAsync(h.tri_orig, sorig.data(), sizeof(int) * NT, cudaMemcpyHostToDevice, st));
    std::vector<int> spos(NT);
    for (int k = 0; k < NT; k++) spos[sorig[k]] = k;
    MK(cudaMemcpyAsync(h.tri_pos, spos.data(), sizeof(int) * NT, cudaMemcpyHostToDevice, st));
    MK(cudaMemcpyAsync(h.tri_mat, smat.data(), sizeof(unsigned) * NT, cudaMemcpyHostToDevice, st));
    // 3: binary radix tree per part
    std::vector<int> ptb(NP), ptc(NP), pnb(NP), nodepart(std::max(nb, 1)), nodebase(std::max(nb, 1));
    for (int p = 0; p < NP; p++) {
        ptb[p] = h.part[p].tri_begin;
        ptc[p] = h.part[p].tri_count;
        pnb[p] = bin_begin[p];
        for (int g = pnb[p]; g < pnb[p] + std::max(ptc[p] - 1, 0); g++) { nodepart[g] = p; nodebase[g] = pnb[p]; }
    }
    std::vector<int4> refs0(std::max(nb, 1), make_int4(0, 0, -1, 0));
    std::vector<int> lp0(NT, -1);
    MK(cudaMemcpyAsync(d_ptb, ptb.data(), sizeof(int) * NP, cudaMemcpyHostToDevice, st));
    MK(cudaMemcpyAsync(d_ptc, ptc.data(), sizeof(int) * NP, cudaMemcpyHostToDevice, st));
    MK(cudaMemcpyAsync(d_pnb, pnb.data(), sizeof(int) * NP, cudaMemcpyHostToDevice, st));
    MK(cudaMemcpyAsync(d_nodepart, nodepart.data(), sizeof(int) * nodepart.size(), cudaMemcpyHostToDevice, st));
    MK(cudaMemcpyAsync(d_nodebase, nodebase.data(), sizeof(int) * nodebase.size(), cudaMemcpyHostToDevice, st));
    MK(cudaMemcpyAsync(node_refs, refs0.data(), sizeof(int4) * refs0.size(), cudaMemcpyHostToDevice, st));
    MK(cudaMemcpyAsync(h.leaf_parent, lp0.data(), sizeof(int) * NT, cudaMemcpyHostToDevice, st));
    MK(launch_karras(keys, d_ptb, d_ptc, d_pnb, NP, nb, d_nodepart, node_refs, h.leaf_parent, st));
    int zero = 0, depth = 0;
    MK(cudaMemcpyAsync(d_depth, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
    MK(launch_depth(node_refs, d_nodebase, nb, d_depth, st));
    MK(cudaMemcpyAsync(&depth, d_depth, sizeof(int), cudaMemcpyDeviceToHost, st));
    MK(cudaStreamSynchronize(st));
    h.max_depth = depth;
    if (depth + 2 > kStack) {
        free_tmp();
        free_mesh(m);
        return fail(ctx, SRP_ERR_MESH, "BVH depth %d exceeds the traversal stack (%d)", depth, kStack);
    }
    // collapse every part's binary tree into 4-wide nodes (host, O(n)); the
    // refit fills the boxes (static parts below, dynamic parts per evaluation)
    {
        std::vector<int4> brefs(std::max(nb, 1));
        MK(cudaMemcpy(brefs.data(), node_refs, sizeof(int4) * std::max(nb, 1), cudaMemcpyDeviceToHost));
        std::vector<int> lp4(NT, -1);
        std::vector<int2> grp(NT, make_int2(kEmptyChild, 0));
        std::vector<float4> tmpl;
        int n4 = 0, depth4 = 0;
        const double pose_err = 1e-14 * h.R;  // bound on the FP64 posing error of a vertex
        for (int r = 0; r < NP; r++) {
            const int p = order[r];
            PartInfo &pi = h.part[p];
            pi.node_begin = n4;
            // each coplanar group is a contiguous run of the part's sorted triangles
            std::map<int, std::array<int, 3>> runs;  // group -> first, last, count
            for (int k = 0; k < pi.tri_count; k++) {
                const int g = tgrp[sorig[pi.tri_begin + k]];
                if (g == 0) continue;
                auto it = runs.find(g);
                if (it == runs.end()) runs[g] = {k, k, 1};
                else { it->second[1] = k; it->second[2]++; }
            }
            std::vector<std::pair<int, int>> pin;
            std::vector<int> pin_g, pin_ref;
            for (auto &kv : runs)
                if (kv.second[1] - kv.second[0] + 1 == kv.second[2]) {
                    pin.push_back({kv.second[0], kv.second[1]});
                    pin_g.push_back(kv.first);
                }
            int d4 = collapse_part(brefs.data() + bin_begin[p], pi.tri_count, pi.tri_begin, svidx, rest, pin, pin_ref,
                                   tmpl, lp4.data() + pi.tri_begin);
            for (size_t i = 0; i < pin.size(); i++) {
                if (pin_ref[i] == kEmptyChild) continue;
                for (int k = pin[i].first; k <= pin[i].second; k++) {
                    const int t = pi.tri_begin + k;
                    const float dev = (float)((tdev[sorig[t]] + pose_err) * 1.001);
                    int bits;
                    memcpy(&bits, &dev, sizeof bits);
                    grp[t] = make_int2(pin_ref[i], bits);
                }
            }
            pi.node_count = (int)(tmpl.size() / kNode4) - n4;
            n4 += pi.node_count;
            depth4 = std::max(depth4, d4);
            if (!pi.dynamic) h.n_static_nodes = n4;
        }
        h.n_dyn_nodes = n4 - h.n_static_nodes;
        for (int p = 0; p < NP; p++) {
            PartInfo &pi = h.part[p];
            pi.dyn_node_off = pi.dynamic ? pi.node_begin - h.n_static_nodes : 0;
        }
        if (3 * depth4 + 1 > kStack) {
            free_tmp();
            free_mesh(m);
            return fail(ctx, SRP_ERR_MESH, "4-wide BVH depth %d exceeds the traversal stack (%d)", depth4, kStack);
        }
        MK(cudaMemcpyAsync(h.leaf_parent, lp4.data(), sizeof(int) * NT, cudaMemcpyHostToDevice, st));
        MK(cudaMemcpyAsync(h.grp, grp.data(), sizeof(int2) * NT, cudaMemcpyHostToDevice, st));
        MK(dmalloc(m->allocs, &h.node_static, (size_t)std::max(h.n_static_nodes, 1) * kNode4));
        MK(dmalloc(m->allocs, &m->node_tmpl_dyn, (size_t)std::max(h.n_dyn_nodes, 1) * kNode4));
        MK(dmalloc(tmp, &cnt_static, (size_t)std::max(h.n_static_nodes, 1)));
        if (h.n_static_nodes > 0)
            MK(cudaMemcpyAsync(h.node_static, tmpl.data(), sizeof(float4) * kNode4 * h.n_static_nodes,
                               cudaMemcpyHostToDevice, st));
        if (h.n_dyn_nodes > 0)
            MK(cudaMemcpyAsync(m->node_tmpl_dyn, tmpl.data() + (size_t)kNode4 * h.n_static_nodes,
                               sizeof(float4) * kNode4 * h.n_dyn_nodes, cudaMemcpyHostToDevice, st));
        MK(cudaStreamSynchronize(st));  // tmpl and lp4 leave scope
    }
    // materials and angles
    std::vector<float2> m32(NM);
    for (int i = 0; i < NM; i++) m32[i] = make_float2((float)D->mat[2 * i], (float)D->mat[2 * i + 1]);
    MK(cudaMemcpyAsync(h.mat32, m32.data(), sizeof(float2) * NM, cudaMemcpyHostToDevice, st));
    MK(cudaMemcpyAsync(h.mat64, D->mat, sizeof(double) * 2 * NM, cudaMemcpyHostToDevice, st));
    MK(cudaMemsetAsync(m->angles_d, 0, sizeof(double) * NP, st));
    MK(cudaMemsetAsync(cnt_static, 0, sizeof(unsigned) * std::max(h.n_static_nodes, 1), st));
    // device copy of the mesh, then the static refit (writes root boxes into it)
    MK(dmalloc(m->allocs, &m->d, 1));
    MK(cudaMemcpyAsync(m->d, &h, sizeof(MeshDev), cudaMemcpyHostToDevice, st));
    MK(launch_refit_static(m->d, h, h.node_static, h.tri_static, cnt_static, &m->d->root_box_static[0][0], st));
    MK(cudaMemcpyAsync(&h.root_box_static[0][0], &m->d->root_box_static[0][0], sizeof(h.root_box_static),
                       cudaMemcpyDeviceToHost, st));
    MK(cudaStreamSynchronize(st));
    free_tmp();
#undef MK
    ctx->meshes.push_back(m);
    *mesh_id = (int32_t)ctx->meshes.size() - 1;
    return SRP_OK;
}

srp_status srp_mesh_free(srp_ctx *ctx, int32_t mesh_id)
{
    Mesh *m = get_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, SRP_ERR_ARG, "bad mesh id %d", mesh_id);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    free_mesh(m);
    ctx->meshes[mesh_id] = nullptr;
    return SRP_OK;
}

srp_status srp_set_panel_angles(srp_ctx *ctx, int32_t mesh_id, int32_t n, const double *rad)
{
    Mesh *m = get_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, SRP_ERR_ARG, "bad mesh id %d", mesh_id);
    if (!rad || n != m->h.n_parts) return fail(ctx, SRP_ERR_ARG, "need %d angles", m->h.n_parts);
    CK(ctx, cudaSetDevice(ctx->device));
    CK(ctx, cudaMemcpyAsync(m->angles_d, rad, sizeof(double) * n,
                            is_device_ptr(rad) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return SRP_OK;
}

srp_status srp_eval_batch(srp_ctx *ctx, int32_t mesh_id, const srp_eval_params *prm, int32_t n,
                          const double *sun_dir_body, const double *quat, const double *sun_dist_au, double *force,
                          double *torque, int32_t *hit_tri)
{
    if (!ctx) return SRP_ERR_ARG;
    ctx->err.clear();
    Mesh *m = get_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, SRP_ERR_STATE, "bad mesh id %d", mesh_id);
    srp_status rc = check_eval_params(ctx, prm);
    if (rc) return rc;
    if (n < 0) return fail(ctx, SRP_ERR_ARG, "n < 0");
    memset(&ctx->last, 0, sizeof ctx->last);
    if (n == 0) return SRP_OK;
    if (!sun_dir_body || !force || !torque) return fail(ctx, SRP_ERR_ARG, "null input or output");
    if (quat && !(m->mass > 0.0)) return fail(ctx, SRP_ERR_ARG, "an attitude quaternion needs the mesh mass > 0");
    CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    EvalPlan pl;
    rc = eval_plan(ctx, m, prm, n, hit_tri != nullptr, pl);
    if (rc) return rc;
    Timing tm(ctx, (prm->flags & SRP_EVAL_TIMING) != 0);
    bool in_dev = is_device_ptr(sun_dir_body);
    bool dist_dev = sun_dist_au && is_device_ptr(sun_dist_au);
    bool f_dev = is_device_ptr(force), t_dev = is_device_ptr(torque);
    bool h_dev = hit_tri && is_device_ptr(hit_tri);
    bool q_dev = quat && is_device_ptr(quat);
    // io: sun (3n) dist (n) force (3n) torque (3n); with a quaternion also q (4n),
    // the body-frame direction (3n) and the body-frame force (3n)
    size_t io_need = (size_t)n * (quat ? 20 : 10);
    CK(ctx, grow(&ctx->io, &ctx->io_cap, io_need, false));
    double *d_sun = in_dev ? const_cast<double *>(sun_dir_body) : ctx->io;
    double *d_dist = sun_dist_au ? (dist_dev ? const_cast<double *>(sun_dist_au) : ctx->io + (size_t)n * 3) : nullptr;
    double *d_f = f_dev ? force : ctx->io + (size_t)n * 4;
    double *d_t = t_dev ? torque : ctx->io + (size_t)n * 7;
    double *d_q = quat ? (q_dev ? const_cast<double *>(quat) : ctx->io + (size_t)n * 10) : nullptr;
    double *d_sb = ctx->io + (size_t)n * 14, *d_fb = ctx->io + (size_t)n * 17;
    int t_in0 = tm.mark(st);
    if (!in_dev) CK(ctx, cudaMemcpyAsync(d_sun, sun_dir_body, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    if (sun_dist_au && !dist_dev)
        CK(ctx, cudaMemcpyAsync(d_dist, sun_dist_au, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    if (quat && !q_dev) CK(ctx, cudaMemcpyAsync(d_q, quat, sizeof(double) * 4 * n, cudaMemcpyHostToDevice, st));
    tm.span(4, t_in0, tm.mark(st));
    CK(ctx, cudaMemsetAsync(ctx->err_flags, 0, sizeof(int), st));
    CK(ctx, cudaMemsetAsync(ctx->stats, 0, 16 * sizeof(unsigned long long), st));
    int64_t launches = 0, trace_launches = 0;
    if (quat) {
        CK(ctx, launch_att_in(n, d_q, d_sun, d_sb, nullptr, nullptr, m->mass, st));
        launches++;
    }
    rc = eval_enqueue(ctx, m, prm, pl, n, quat ? d_sb : d_sun, d_dist, quat ? d_fb : d_f, d_t, hit_tri, h_dev, tm,
                      launches, trace_launches);
    if (rc) return rc;
    if (quat) {
        CK(ctx, launch_att_out(n, d_q, d_fb, d_f, m->mass, st));
        launches++;
    }
    int t_out0 = tm.mark(st);
    if (!f_dev) CK(ctx, cudaMemcpyAsync(force, d_f, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
    if (!t_dev) CK(ctx, cudaMemcpyAsync(torque, d_t, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
    tm.span(4, t_out0, tm.mark(st));
    int flags = 0;
    unsigned long long stats[16];
    CK(ctx, cudaMemcpyAsync(&flags, ctx->err_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaMemcpyAsync(stats, ctx->stats, sizeof stats, cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaStreamSynchronize(st));
    fill_stats(ctx->last, stats);
    ctx->last.launches = launches;
    ctx->last.trace_launches = trace_launches;
    tm.collect(ctx->last);
    if (flags & kFlagTimeout) return fail(ctx, SRP_ERR_TIMEOUT, "a work-queue wait gave up");
    if (flags & kFlagStack) return fail(ctx, SRP_ERR_STACK, "traversal stack bound reached");
    return SRP_OK;
}

srp_status srp_propagate(srp_ctx *ctx, int32_t mesh_id, const srp_prop_params *p, int32_t n, const double *y0,
                         const double *t0_t1, double *y1, srp_prop_stats *stats, double *h_log, int64_t h_cap)
{
    if (!ctx) return SRP_ERR_ARG;
    ctx->err.clear();
    Mesh *m = get_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, SRP_ERR_STATE, "bad mesh id %d", mesh_id);
    if (!p) return fail(ctx, SRP_ERR_ARG, "null params");
    const bool spad = p->spad_table != nullptr;
    srp_status rc = spad ? check_spad_grid(ctx, &p->spad_grid) : check_eval_params(ctx, &p->eval);
    if (rc) return rc;
    if (n <= 0 || !y0 || !t0_t1 || !y1) return fail(ctx, SRP_ERR_ARG, "need n > 0, y0, t0_t1 and y1");
    if (p->method != SRP_RKF78 && p->method != SRP_RK4) return fail(ctx, SRP_ERR_ARG, "bad method");
    if (p->central != SRP_CENTRAL_EARTH && p->central != SRP_CENTRAL_SUN) return fail(ctx, SRP_ERR_ARG, "bad central body");
    if (p->attitude != SRP_ATT_LVLH && p->attitude != SRP_ATT_INERTIAL) return fail(ctx, SRP_ERR_ARG, "bad attitude");
    if (!(p->h0 > 0.0) || !(p->h_min >= 0.0) || p->max_steps <= 0) return fail(ctx, SRP_ERR_ARG, "bad step settings");
    if (p->method == SRP_RKF78 && (!(p->rtol > 0.0) || !(p->atol_pos > 0.0) || !(p->atol_vel > 0.0)))
        return fail(ctx, SRP_ERR_ARG, "tolerances must be > 0");
    if (p->srp && !(m->mass > 0.0)) return fail(ctx, SRP_ERR_ARG, "mesh mass must be > 0 for SRP");
    if (h_log && h_cap <= 0) return fail(ctx, SRP_ERR_ARG, "h_cap must be > 0 with h_log");
    CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    memset(&ctx->last, 0, sizeof ctx->last);
    EvalPlan pl;
    if (!spad) {
        rc = eval_plan(ctx, m, &p->eval, n, false, pl);
        if (rc) return rc;
    }
    // device buffers (grown, kept by the context)
    size_t need = (size_t)n * (3 + 1 + 3 + 3 + 6 + 2);
    CK(ctx, grow(&ctx->prop_io, &ctx->prop_io_cap, need, false));
    CK(ctx, grow(&ctx->prop_state, &ctx->prop_state_cap, (size_t)n, false));
    if (h_log) CK(ctx, grow(&ctx->prop_hlog, &ctx->prop_hlog_cap, (size_t)n * h_cap, false));
    double *d_sun = ctx->prop_io, *d_dist = d_sun + 3 * (size_t)n, *d_f = d_dist + n, *d_t = d_f + 3 * (size_t)n;
    double *d_y0 = d_t + 3 * (size_t)n, *d_t01 = d_y0 + 6 * (size_t)n;
    CK(ctx, cudaMemcpyAsync(d_y0, y0, sizeof(double) * 6 * n, cudaMemcpyDefault, st));
    CK(ctx, cudaMemcpyAsync(d_t01, t0_t1, sizeof(double) * 2 * n, cudaMemcpyDefault, st));
    CK(ctx, cudaMemsetAsync(ctx->err_flags, 0, sizeof(int), st));
    CK(ctx, cudaMemsetAsync(ctx->stats, 0, 16 * sizeof(unsigned long long), st));
    CK(ctx, cudaMemsetAsync(ctx->prop_done, 0, sizeof(int), st));
    PropState *S = ctx->prop_state;
    PropDev P = prop_dev(p, m);
    if (spad) {
        // the SPAD table replaces the ray tracer (Sec. 4.2): staged once on the device
        const size_t nt = (size_t)p->spad_grid.n_az * p->spad_grid.n_el * 6;
        CK(ctx, grow(&ctx->spad_buf, &ctx->spad_cap, nt, false));
        CK(ctx, cudaMemcpyAsync(ctx->spad_buf, p->spad_table, sizeof(double) * nt, cudaMemcpyDefault, st));
        P.spad = spad_dev(&p->spad_grid, ctx->spad_buf);
    }
    const bool trace = p->srp && !spad;
    CK(ctx, launch_prop_init(S, n, d_y0, d_t01, P, nullptr, ctx->prop_done, st));
    if (p->h_replay && p->n_replay > 0) {
        if (p->method != SRP_RKF78) return fail(ctx, SRP_ERR_ARG, "step replay needs SRP_RKF78");
        CK(ctx, grow(&ctx->prop_replay, &ctx->prop_replay_cap, (size_t)n * p->n_replay, false));
        CK(ctx, cudaMemcpyAsync(ctx->prop_replay, p->h_replay, sizeof(double) * n * p->n_replay, cudaMemcpyDefault, st));
        P.h_replay = ctx->prop_replay;
        P.n_replay = p->n_replay;
    }
    const int nstage = p->method == SRP_RK4 ? 4 : 13;
    Timing off(ctx, false);
    int64_t launches = 0, trace_launches = 0;
    if (p->host_loop) {
        // the same kernels, issued stage by stage with the host waiting for each
        // stage's SRP result, as a host-side integrator calling a GPU force model would
        int done = 0;
        for (int64_t step = 0; step <= p->max_steps + 1; step++) {
            CK(ctx, cudaMemcpyAsync(&done, ctx->prop_done, sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(ctx, cudaStreamSynchronize(st));
            if (done >= n) break;
            for (int sg = 0; sg < nstage; sg++) {
                CK(ctx, launch_prop_stage(S, n, P, sg, d_sun, d_dist, st));
                if (trace) {
                    srp_status erc = eval_enqueue(ctx, m, &p->eval, pl, n, d_sun, d_dist, d_f, d_t, nullptr, false,
                                                  off, launches, trace_launches);
                    if (erc) return erc;
                }
                CK(ctx, cudaStreamSynchronize(st));
                CK(ctx, launch_prop_accel(S, n, P, sg, d_f, st, d_sun, d_dist));
            }
            CK(ctx, launch_prop_control(S, n, P, ctx->prop_done, h_log ? ctx->prop_hlog : nullptr, h_cap, st));
        }
        return finish_propagate(ctx, n, S, y1, stats, h_log, h_cap);
    }
    // capture one step into a graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    CK(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    srp_status crc = SRP_OK;
    if (!trace) {
        // no ray-traced evaluation between the stages: the whole step is one kernel
        if (launch_prop_step(S, n, P, d_sun, d_dist, ctx->prop_done, h_log ? ctx->prop_hlog : nullptr, h_cap, st) !=
            cudaSuccess)
            crc = SRP_ERR_CUDA;
    } else {
        // a step starts from its first stage's state, made by the previous step's
        // last launch (or, before the first step, by the launch after the capture)
        for (int sg = 0; sg < nstage && crc == SRP_OK; sg++) {
            crc = eval_enqueue(ctx, m, &p->eval, pl, n, d_sun, d_dist, d_f, d_t, nullptr, false, off, launches,
                               trace_launches);
            if (crc == SRP_OK && launch_prop_next(S, n, P, sg, d_f, d_sun, d_dist, ctx->prop_done,
                                                  h_log ? ctx->prop_hlog : nullptr, h_cap, st) != cudaSuccess)
                crc = SRP_ERR_CUDA;
        }
    }
    cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (crc != SRP_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return crc != SRP_OK ? crc : fail(ctx, SRP_ERR_CUDA, "step capture failed: %s", cudaGetErrorString(ce));
    }
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(ctx, SRP_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
    if (trace && launch_prop_stage(S, n, P, 0, d_sun, d_dist, st) != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        return fail(ctx, SRP_ERR_CUDA, "first stage launch failed");
    }
    // relaunch until every trajectory is done.  Each round launches about as many
    // steps as the furthest trajectory still needs at its current step size
    // (at most `poll`), so finished work is rarely repeated; finished and
    // shadowed trajectories skip their SRP evaluations anyway.
    const int poll_max = p->poll > 0 ? p->poll : 16;
    const int64_t max_rounds = p->max_steps + 2;
    int done = 0;
    std::vector<PropState> peek(n);
    int launch = 1;
    for (int64_t round = 0; round < max_rounds; round++) {
        CK(ctx, cudaMemcpyAsync(&done, ctx->prop_done, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(ctx, cudaMemcpyAsync(peek.data(), S, sizeof(PropState) * n, cudaMemcpyDeviceToHost, st));
        cudaError_t se = cudaStreamSynchronize(st);
        if (se != cudaSuccess) { cudaGraphExecDestroy(exec); return fail(ctx, SRP_ERR_CUDA, "%s", cudaGetErrorString(se)); }
        if (done >= n) break;
        double need = 1.0;
        for (int i = 0; i < n; i++) {
            const PropState &X = peek[i];
            if (X.done) continue;
            double r = P.n_replay > 0 ? (double)(P.n_replay - X.steps) : (X.t1 - X.t) / fmax(X.h, 1e-300);
            need = fmax(need, r);
        }
        launch = (int)std::min<double>(poll_max, std::max(1.0, std::ceil(need)));
        for (int k = 0; k < launch; k++) {
            se = cudaGraphLaunch(exec, st);
            if (se != cudaSuccess) { cudaGraphExecDestroy(exec); return fail(ctx, SRP_ERR_CUDA, "%s", cudaGetErrorString(se)); }
        }
    }
    cudaGraphExecDestroy(exec);
    return finish_propagate(ctx, n, S, y1, stats, h_log, h_cap);
}

srp_status srp_spad_build(srp_ctx *ctx, int32_t mesh_id, const srp_eval_params *prm, const srp_spad_grid *g,
                          double *table)
{
    if (!ctx) return SRP_ERR_ARG;
    ctx->err.clear();
    srp_status rc = check_spad_grid(ctx, g);
    if (rc) return rc;
    if (!prm || !table) return fail(ctx, SRP_ERR_ARG, "null params or table");
    if (!get_mesh(ctx, mesh_id)) return fail(ctx, SRP_ERR_STATE, "bad mesh id %d", mesh_id);
    CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const int n = g->n_az * g->n_el;
    CK(ctx, grow(&ctx->spad_buf, &ctx->spad_cap, (size_t)n * 9, false));
    double *d_dir = ctx->spad_buf, *d_f = d_dir + 3 * (size_t)n, *d_t = d_f + 3 * (size_t)n;
    CK(ctx, launch_spad_dirs(spad_dev(g, nullptr), d_dir, st));
    // one evaluation per sample direction at 1 AU, through the evaluation pipeline
    rc = srp_eval_batch(ctx, mesh_id, prm, n, d_dir, nullptr, nullptr, d_f, d_t, nullptr);
    if (rc) return rc;
    // [n][3] force and torque interleaved into the table's [n][6]
    const size_t v3 = 3 * sizeof(double), v6 = 6 * sizeof(double);
    CK(ctx, cudaMemcpy2DAsync(table, v6, d_f, v3, v3, n, cudaMemcpyDefault, st));
    CK(ctx, cudaMemcpy2DAsync(table + 3, v6, d_t, v3, v3, n, cudaMemcpyDefault, st));
    CK(ctx, cudaStreamSynchronize(st));
    return SRP_OK;
}

srp_status srp_spad_eval(srp_ctx *ctx, const srp_spad_grid *g, const double *table, int32_t n,
                         const double *sun_dir_body, const double *sun_dist_au, double *force, double *torque)
{
    if (!ctx) return SRP_ERR_ARG;
    ctx->err.clear();
    srp_status rc = check_spad_grid(ctx, g);
    if (rc) return rc;
    if (n < 0) return fail(ctx, SRP_ERR_ARG, "n < 0");
    if (n == 0) return SRP_OK;
    if (!table || !sun_dir_body || !force || !torque) return fail(ctx, SRP_ERR_ARG, "null table, input or output");
    CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const size_t nt = (size_t)g->n_az * g->n_el * 6, n3 = 3 * (size_t)n;
    const bool tab_dev = is_device_ptr(table), in_dev = is_device_ptr(sun_dir_body);
    const bool dist_dev = sun_dist_au && is_device_ptr(sun_dist_au);
    const bool f_dev = is_device_ptr(force), t_dev = is_device_ptr(torque);
    const size_t need = (tab_dev ? 0 : nt) + (in_dev ? 0 : n3) + (sun_dist_au && !dist_dev ? (size_t)n : 0) +
                        (f_dev ? 0 : n3) + (t_dev ? 0 : n3);
    CK(ctx, grow(&ctx->spad_buf, &ctx->spad_cap, need, false));
    double *q = ctx->spad_buf;
    const double *d_tab = table, *d_dir = sun_dir_body, *d_dist = sun_dist_au;
    if (!tab_dev) { CK(ctx, cudaMemcpyAsync(q, table, sizeof(double) * nt, cudaMemcpyHostToDevice, st)); d_tab = q; q += nt; }
    if (!in_dev) { CK(ctx, cudaMemcpyAsync(q, sun_dir_body, sizeof(double) * n3, cudaMemcpyHostToDevice, st)); d_dir = q; q += n3; }
    if (sun_dist_au && !dist_dev) {
        CK(ctx, cudaMemcpyAsync(q, sun_dist_au, sizeof(double) * n, cudaMemcpyHostToDevice, st));
        d_dist = q;
        q += n;
    }
    double *d_f = force, *d_t = torque;
    if (!f_dev) { d_f = q; q += n3; }
    if (!t_dev) { d_t = q; q += n3; }
    CK(ctx, launch_spad_eval(spad_dev(g, d_tab), n, d_dir, d_dist, d_f, d_t, st));
    if (!f_dev) CK(ctx, cudaMemcpyAsync(force, d_f, sizeof(double) * n3, cudaMemcpyDeviceToHost, st));
    if (!t_dev) CK(ctx, cudaMemcpyAsync(torque, d_t, sizeof(double) * n3, cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaStreamSynchronize(st));
    return SRP_OK;
}

srp_status srp_set_memory_limit(srp_ctx *ctx, uint64_t bytes)
{
    if (!ctx) return SRP_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mem_mu);
    g_mem_limit = (size_t)bytes;
    return SRP_OK;
}

srp_status srp_memory_usage(srp_ctx *ctx, uint64_t *used, uint64_t *limit)
{
    if (!ctx || !used || !limit) return SRP_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mem_mu);
    *used = g_mem_used;
    *limit = g_mem_limit;
    return SRP_OK;
}

srp_status srp_sort_pairs(srp_ctx *ctx, int32_t n, uint64_t *keys, int32_t *vals, int32_t key_bits)
{
    if (!ctx) return SRP_ERR_ARG;
    ctx->err.clear();
    if (n < 0 || (n > 0 && (!keys || !vals)) || key_bits < 1 || key_bits > 64)
        return fail(ctx, SRP_ERR_ARG, "need n >= 0, keys, vals and 1 <= key_bits <= 64");
    if (n <= 1) return SRP_OK;
    CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    struct Tmp {
        std::vector<void *> v;
        ~Tmp() { for (void *q : v) dfree(q); }
    } tmp;
    const size_t sc = radix_sort_scratch_ints(n);
    unsigned long long *k0, *k1;
    int *v0, *v1, *scr;
    CK(ctx, dmalloc(tmp.v, &k0, (size_t)n));
    CK(ctx, dmalloc(tmp.v, &k1, (size_t)n));
    CK(ctx, dmalloc(tmp.v, &v0, (size_t)n));
    CK(ctx, dmalloc(tmp.v, &v1, (size_t)n));
    CK(ctx, dmalloc(tmp.v, &scr, sc));
    CK(ctx, cudaMemcpyAsync(k0, keys, sizeof(unsigned long long) * n, cudaMemcpyDefault, st));
    CK(ctx, cudaMemcpyAsync(v0, vals, sizeof(int) * n, cudaMemcpyDefault, st));
    CK(ctx, radix_sort_pairs(k0, v0, k1, v1, n, 0, (key_bits + 7) / 8 * 8, scr, sc, st));
    CK(ctx, cudaMemcpyAsync(keys, k0, sizeof(unsigned long long) * n, cudaMemcpyDefault, st));
    CK(ctx, cudaMemcpyAsync(vals, v0, sizeof(int) * n, cudaMemcpyDefault, st));
    CK(ctx, cudaStreamSynchronize(st));
    return SRP_OK;
}

srp_status srp_mesh_check(srp_ctx *ctx, int32_t mesh_id, const double *sun_dir_body, int64_t *report)
{
    if (!ctx) return SRP_ERR_ARG;
    ctx->err.clear();
    if (!report) return fail(ctx, SRP_ERR_ARG, "null report");
    Mesh *m = get_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, SRP_ERR_STATE, "bad mesh id %d", mesh_id);
    double s[3] = {0.0, 0.0, 1.0};
    if (sun_dir_body) for (int k = 0; k < 3; k++) s[k] = sun_dir_body[k];
    // one evaluation poses the mesh and refits its tree in slot 0 (one slot, one lane)
    srp_eval_params prm{};
    prm.N = 1;
    prm.bounces = 0;
    prm.P0 = 4.56e-6;
    prm.eps_rel = 1e-9;
    prm.panel_mode = SRP_PANELS_TRACK;
    prm.flags = SRP_EVAL_TRAVERSE;
    double F[3], T[3];
    srp_status rc = srp_eval_batch(ctx, mesh_id, &prm, 1, s, nullptr, nullptr, F, T, nullptr);
    if (rc) return rc;
    cudaStream_t st = ctx->stream;
    struct Tmp {
        std::vector<void *> v;
        ~Tmp() { for (void *q : v) dfree(q); }
    } tmp;
    const int nt = m->h.n_tris;
    int *seen;
    unsigned long long *rep;
    CK(ctx, dmalloc(tmp.v, &seen, (size_t)nt));
    CK(ctx, dmalloc(tmp.v, &rep, (size_t)8));
    CK(ctx, cudaMemsetAsync(seen, 0, sizeof(int) * nt, st));
    CK(ctx, cudaMemsetAsync(rep, 0, sizeof(unsigned long long) * 8, st));
    CK(ctx, launch_bvh_check(ctx->tctx, m->h.n_parts, seen, rep, st));
    std::vector<int> hs(nt);
    unsigned long long hr[8];
    CK(ctx, cudaMemcpyAsync(hs.data(), seen, sizeof(int) * nt, cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaMemcpyAsync(hr, rep, sizeof hr, cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaStreamSynchronize(st));
    int64_t bad = 0;
    for (int c : hs) bad += c != 1;
    report[0] = (int64_t)hr[0];
    report[1] = bad;
    for (int k = 2; k < 6; k++) report[k] = (int64_t)hr[k];
    report[6] = nt;
    report[7] = m->h.n_parts;
    return SRP_OK;
}

srp_status srp_eval_stats_get(srp_ctx *ctx, srp_eval_stats *out)
{
    if (!ctx || !out) return SRP_ERR_ARG;
    *out = ctx->last;
    return SRP_OK;
}

srp_status srp_set_materials(srp_ctx *ctx, int32_t mesh_id, int32_t n_mats, const double *mat)
{
    if (!ctx) return SRP_ERR_ARG;
    ctx->err.clear();
    Mesh *m = get_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, SRP_ERR_ARG, "bad mesh id %d", mesh_id);
    if (!mat || n_mats != m->h.n_mats) return fail(ctx, SRP_ERR_ARG, "need %d materials", m->h.n_mats);
    CK(ctx, cudaSetDevice(ctx->device));
    std::vector<double> hm((size_t)2 * n_mats);
    CK(ctx, cudaMemcpy(hm.data(), mat, sizeof(double) * hm.size(), cudaMemcpyDefault));
    std::vector<float2> m32(n_mats);
    for (int i = 0; i < n_mats; i++) {
        double rs = hm[2 * i], rd = hm[2 * i + 1];
        if (!(rs >= 0.0 && rd >= 0.0 && rs + rd <= 1.0 + 1e-12))
            return fail(ctx, SRP_ERR_MESH, "material %d coefficients (%g, %g) outside [0,1] or sum > 1", i, rs, rd);
        m32[i] = make_float2((float)rs, (float)rd);
    }
    cudaStream_t st = ctx->stream;
    CK(ctx, cudaMemcpyAsync(m->h.mat32, m32.data(), sizeof(float2) * n_mats, cudaMemcpyHostToDevice, st));
    CK(ctx, cudaMemcpyAsync(m->h.mat64, hm.data(), sizeof(double) * hm.size(), cudaMemcpyHostToDevice, st));
    CK(ctx, cudaStreamSynchronize(st));
    return SRP_OK;
}

srp_status srp_grad(srp_ctx *ctx, int32_t mesh_id, const srp_eval_params *prm, int32_t n, const double *sun_dir_body,
                    const double *quat, const double *sun_dist_au, const double *g_force, const double *g_torque,
                    double *force, double *torque, double *g_sun, double *g_dist, double *g_mat, double *g_angle,
                    double *g_quat)
{
    if (!ctx) return SRP_ERR_ARG;
    ctx->err.clear();
    Mesh *m = get_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, SRP_ERR_STATE, "bad mesh id %d", mesh_id);
    srp_status rc = check_eval_params(ctx, prm);
    if (rc) return rc;
    if (prm->n_diffuse != 0) return fail(ctx, SRP_ERR_ARG, "srp_grad takes no diffuse rays (n_diffuse = 0)");
    if (n < 0) return fail(ctx, SRP_ERR_ARG, "n < 0");
    if (g_dist && !sun_dist_au) return fail(ctx, SRP_ERR_ARG, "g_dist needs sun_dist_au");
    if (g_quat && !quat) return fail(ctx, SRP_ERR_ARG, "g_quat needs quat");
    if (quat && !(m->mass > 0.0)) return fail(ctx, SRP_ERR_ARG, "an attitude quaternion needs the mesh mass > 0");
    memset(&ctx->last, 0, sizeof ctx->last);
    const int NM2 = 2 * m->h.n_mats, NP = m->h.n_parts, GE = NM2 + NP;
    CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    if (n == 0) {
        // empty batch: the summed gradients are zero
        std::vector<double> z((size_t)GE, 0.0);
        if (g_mat) CK(ctx, cudaMemcpy(g_mat, z.data(), sizeof(double) * NM2, cudaMemcpyDefault));
        if (g_angle) CK(ctx, cudaMemcpy(g_angle, z.data(), sizeof(double) * NP, cudaMemcpyDefault));
        return SRP_OK;
    }
    if (!sun_dir_body || !g_force || !g_torque) return fail(ctx, SRP_ERR_ARG, "null input or cotangent");
    EvalPlan pl;
    rc = eval_plan(ctx, m, prm, n, false, pl, true);
    if (rc) return rc;
    // device staging: inputs, cotangents, outputs, per-evaluation terms, batch sums
    const size_t n3 = (size_t)n * 3;
    size_t off_sun = 0, off_dist = n3, off_gf = off_dist + n, off_gt = off_gf + n3, off_f = off_gt + n3,
           off_t = off_f + n3, off_gs = off_t + n3, off_gd = off_gs + n3, off_ge = off_gd + n,
           off_sum = off_ge + (size_t)n * GE, off_q = off_sum + GE, off_gq = off_q + 4 * (size_t)n,
           off_sb = off_gq + 4 * (size_t)n, off_gfb = off_sb + n3, off_fb = off_gfb + n3, off_gsb = off_fb + n3,
           need = quat ? off_gsb + n3 : off_q;
    CK(ctx, grow(&ctx->gio, &ctx->gio_cap, need, false));
    double *G = ctx->gio;
    struct In {
        const double *src;
        size_t off, count;
    } ins[5] = {{sun_dir_body, off_sun, n3}, {sun_dist_au, off_dist, (size_t)n}, {g_force, off_gf, n3},
                {g_torque, off_gt, n3}, {quat, off_q, 4 * (size_t)n}};
    const double *dev[5];
    for (int k = 0; k < 5; k++) {
        if (!ins[k].src) { dev[k] = nullptr; continue; }
        if (is_device_ptr(ins[k].src)) { dev[k] = ins[k].src; continue; }
        CK(ctx, cudaMemcpyAsync(G + ins[k].off, ins[k].src, sizeof(double) * ins[k].count, cudaMemcpyHostToDevice, st));
        dev[k] = G + ins[k].off;
    }
    CK(ctx, cudaMemsetAsync(ctx->err_flags, 0, sizeof(int), st));
    CK(ctx, cudaMemsetAsync(ctx->stats, 0, 16 * sizeof(unsigned long long), st));
    int64_t launches = 0, trace_launches = 0;
    // with a quaternion the evaluation runs on the body-frame direction and the
    // body-frame force cotangent; the attitude is differentiated around it
    const double *e_sun = dev[0], *e_gf = dev[2];
    double *e_f = G + off_f, *e_gs = G + off_gs;
    if (quat) {
        CK(ctx, launch_att_in(n, dev[4], dev[0], G + off_sb, dev[2], G + off_gfb, m->mass, st));
        launches++;
        e_sun = G + off_sb; e_gf = G + off_gfb; e_f = G + off_fb; e_gs = G + off_gsb;
    }
    AdjBatch ab{e_sun, dev[1], e_gf, dev[3], e_gs, g_dist ? G + off_gd : nullptr, G + off_ge, prm->panel_mode};
    Timing tm(ctx, false);
    rc = eval_enqueue(ctx, m, prm, pl, n, e_sun, dev[1], e_f, G + off_t, nullptr, false, tm, launches,
                      trace_launches, &ab);
    if (rc) return rc;
    CK(ctx, launch_adj_sum(G + off_ge, n, m->h.n_mats, NP, G + off_sum, G + off_sum + NM2, st));
    launches++;
    if (quat) {
        CK(ctx, launch_att_grad(n, dev[4], dev[0], e_f, dev[2], e_gs, G + off_gs, G + off_gq, m->mass, st));
        CK(ctx, launch_att_out(n, dev[4], e_f, G + off_f, m->mass, st));
        launches += 2;
    }
    struct Out {
        double *dst;
        size_t off, count;
    } outs[7] = {{force, off_f, n3}, {torque, off_t, n3}, {g_sun, off_gs, n3}, {g_dist, off_gd, (size_t)n},
                 {g_mat, off_sum, (size_t)NM2}, {g_angle, off_sum + NM2, (size_t)NP}, {g_quat, off_gq, 4 * (size_t)n}};
    for (auto &o : outs)
        if (o.dst) CK(ctx, cudaMemcpyAsync(o.dst, G + o.off, sizeof(double) * o.count, cudaMemcpyDefault, st));
    int flags = 0;
    unsigned long long stats[16];
    CK(ctx, cudaMemcpyAsync(&flags, ctx->err_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaMemcpyAsync(stats, ctx->stats, sizeof stats, cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaStreamSynchronize(st));
    fill_stats(ctx->last, stats);
    ctx->last.launches = launches;
    ctx->last.trace_launches = trace_launches;
    if (flags & kFlagTimeout) return fail(ctx, SRP_ERR_TIMEOUT, "a work-queue wait gave up");
    if (flags & kFlagStack) return fail(ctx, SRP_ERR_STACK, "traversal stack bound reached");
    return SRP_OK;
}

srp_status srp_prop_grad(srp_ctx *ctx, int32_t mesh_id, const srp_prop_params *p, int32_t n, const double *y0,
                         const double *t0_t1, const double *g_y1, int32_t ckpt_every, double *y1, double *g_y0,
                         double *g_mat, double *g_angle, double *g_q, srp_prop_stats *stats)
{
    if (!ctx) return SRP_ERR_ARG;
    ctx->err.clear();
    Mesh *m = get_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, SRP_ERR_STATE, "bad mesh id %d", mesh_id);
    if (!p) return fail(ctx, SRP_ERR_ARG, "null params");
    srp_status rc = check_eval_params(ctx, &p->eval);
    if (rc) return rc;
    if (n <= 0 || !y0 || !t0_t1 || !g_y1) return fail(ctx, SRP_ERR_ARG, "need n > 0, y0, t0_t1 and g_y1");
    if (p->method != SRP_RK4) return fail(ctx, SRP_ERR_ARG, "the propagation adjoint needs SRP_RK4 (fixed steps)");
    if (p->h_replay && p->n_replay > 0) return fail(ctx, SRP_ERR_ARG, "step replay is not differentiated");
    if (p->spad_table) return fail(ctx, SRP_ERR_ARG, "the propagation adjoint traces rays; no SPAD table");
    if (p->eval.n_diffuse != 0) return fail(ctx, SRP_ERR_ARG, "the propagation adjoint takes no diffuse rays");
    if (p->central != SRP_CENTRAL_EARTH && p->central != SRP_CENTRAL_SUN) return fail(ctx, SRP_ERR_ARG, "bad central body");
    if (p->attitude != SRP_ATT_LVLH && p->attitude != SRP_ATT_INERTIAL) return fail(ctx, SRP_ERR_ARG, "bad attitude");
    if (!(p->h0 > 0.0) || p->max_steps <= 0) return fail(ctx, SRP_ERR_ARG, "bad step settings");
    if (ckpt_every < 1) return fail(ctx, SRP_ERR_ARG, "ckpt_every must be >= 1");
    if (p->srp && !(m->mass > 0.0)) return fail(ctx, SRP_ERR_ARG, "mesh mass must be > 0 for SRP");
    CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    memset(&ctx->last, 0, sizeof ctx->last);
    // every trajectory takes the same number of steps
    std::vector<double> t01h((size_t)2 * n);
    CK(ctx, cudaMemcpy(t01h.data(), t0_t1, sizeof(double) * 2 * n, cudaMemcpyDefault));
    const int64_t K = rk4_steps(t01h[0], t01h[1], p->h0, p->max_steps);
    if (K < 0) return fail(ctx, SRP_ERR_STEP, "the arc needs more than max_steps steps");
    for (int i = 1; i < n; i++)
        if (rk4_steps(t01h[2 * i], t01h[2 * i + 1], p->h0, p->max_steps) != K)
            return fail(ctx, SRP_ERR_ARG, "trajectory %d takes a different number of steps", i);
    const int C = (int)std::min<int64_t>(ckpt_every, std::max<int64_t>(K, 1));
    const int64_t nck = K > 0 ? (K + C - 1) / C : 0;
    EvalPlan pl;
    rc = eval_plan(ctx, m, &p->eval, n, false, pl, true);
    if (rc) return rc;
    const int NM2 = 2 * m->h.n_mats, NP = m->h.n_parts, GE = NM2 + NP;
    const size_t R = pl.R, nseg = pl.nseg, n3 = (size_t)n * 3;
    // device buffers
    const size_t rec_count = (size_t)C * 4 * n;
    CK(ctx, grow(&ctx->arc_hits, &ctx->arc_hits_cap, p->srp ? rec_count * R * nseg : 1, false));
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
    const size_t o_state = take(sizeof(PropState) * n), o_adj = take(sizeof(PropAdj) * n),
                 o_ckpt = take(sizeof(double) * 7 * n * std::max<int64_t>(nck, 1)),
                 o_rec = take(sizeof(StageRec) * rec_count), o_rsun = take(sizeof(double) * 3 * rec_count),
                 o_rdist = take(sizeof(double) * rec_count), o_io = take(sizeof(double) * (8 * n3 + 2 * n + 8)),
                 o_ge = take(sizeof(double) * ((size_t)n * GE + GE + 4)), o_t01 = take(sizeof(double) * 2 * n);
    CK(ctx, grow(&ctx->arc_buf, &ctx->arc_buf_cap, off, false));
    unsigned char *B = ctx->arc_buf;
    PropState *S = reinterpret_cast<PropState *>(B + o_state);
    PropAdj *A = reinterpret_cast<PropAdj *>(B + o_adj);
    double *ck = reinterpret_cast<double *>(B + o_ckpt);
    StageRec *rec = reinterpret_cast<StageRec *>(B + o_rec);
    double *rsun = reinterpret_cast<double *>(B + o_rsun), *rdist = reinterpret_cast<double *>(B + o_rdist);
    double *io = reinterpret_cast<double *>(B + o_io);
    double *d_sun = io, *d_f = io + n3, *d_t = io + 2 * n3, *gF = io + 3 * n3, *gT = io + 4 * n3,
           *gS = io + 5 * n3, *d_y0 = io + 6 * n3, *d_dist = io + 8 * n3, *gD = d_dist + n;
    double *ge = reinterpret_cast<double *>(B + o_ge), *acc = ge + (size_t)n * GE, *qsum = acc + GE;
    double *d_t01 = reinterpret_cast<double *>(B + o_t01);
    CK(ctx, cudaMemcpyAsync(d_y0, y0, sizeof(double) * 6 * n, cudaMemcpyDefault, st));
    CK(ctx, cudaMemcpyAsync(d_t01, t0_t1, sizeof(double) * 2 * n, cudaMemcpyDefault, st));
    CK(ctx, cudaMemsetAsync(gT, 0, sizeof(double) * n3, st));
    CK(ctx, cudaMemsetAsync(acc, 0, sizeof(double) * (GE + 4), st));
    CK(ctx, cudaMemsetAsync(A, 0, sizeof(PropAdj) * n, st));
    CK(ctx, cudaMemsetAsync(ctx->err_flags, 0, sizeof(int), st));
    CK(ctx, cudaMemsetAsync(ctx->stats, 0, 16 * sizeof(unsigned long long), st));
    CK(ctx, cudaMemsetAsync(ctx->prop_done, 0, sizeof(int), st));
    const PropDev P = prop_dev(p, m);
    CK(ctx, launch_prop_init(S, n, d_y0, d_t01, P, nullptr, ctx->prop_done, st));
    Timing off_t(ctx, false);
    int64_t launches = 1, trace_launches = 0;
    // one RK4 step; with hrec != null every stage's hits and state are recorded at step j of the segment
    auto step = [&](int64_t j, bool record) -> srp_status {
        for (int sg = 0; sg < 4; sg++) {
            CK(ctx, launch_prop_stage(S, n, P, sg, d_sun, d_dist, st));
            const size_t k = (size_t)j * 4 + sg;
            if (p->srp) {
                int32_t *hrec = record ? ctx->arc_hits + k * n * R * nseg : nullptr;
                srp_status e = eval_enqueue(ctx, m, &p->eval, pl, n, d_sun, d_dist, d_f, d_t, hrec, record, off_t,
                                            launches, trace_launches);
                if (e) return e;
            }
            CK(ctx, launch_prop_accel(S, n, P, sg, d_f, st));
            launches += 2;
            if (record) {
                CK(ctx, launch_prop_record(S, n, d_sun, d_dist, d_f, rec + k * n, rsun + k * 3 * n, rdist + k * n, st));
                launches++;
            }
        }
        CK(ctx, launch_prop_control(S, n, P, ctx->prop_done, nullptr, 0, st));
        launches++;
        return SRP_OK;
    };
    // forward, saving a checkpoint at the start of every segment
    for (int64_t c = 0; c < nck; c++) {
        CK(ctx, launch_prop_ckpt(S, n, ck + (size_t)c * 7 * n, true, p->h0, st));
        const int64_t Ks = std::min<int64_t>(C, K - c * C);
        for (int64_t j = 0; j < Ks; j++)
            if ((rc = step(j, false))) return rc;
    }
    std::vector<PropState> fin(n);
    CK(ctx, cudaMemcpyAsync(fin.data(), S, sizeof(PropState) * n, cudaMemcpyDeviceToHost, st));
    // reverse: lam = g_y1, then segment by segment from the end
    std::vector<PropAdj> a0(n);
    {
        std::vector<double> g1((size_t)6 * n);
        CK(ctx, cudaMemcpy(g1.data(), g_y1, sizeof(double) * 6 * n, cudaMemcpyDefault));
        for (int i = 0; i < n; i++) {
            memset(&a0[i], 0, sizeof(PropAdj));
            for (int k = 0; k < 6; k++) a0[i].lam[k] = g1[6 * (size_t)i + k];
        }
        CK(ctx, cudaMemcpyAsync(A, a0.data(), sizeof(PropAdj) * n, cudaMemcpyHostToDevice, st));
        CK(ctx, cudaStreamSynchronize(st));  // a0 leaves scope
    }
    AdjBatch ab{d_sun, nullptr, gF, gT, gS, gD, ge, p->eval.panel_mode};
    for (int64_t c = nck - 1; c >= 0; c--) {
        CK(ctx, launch_prop_ckpt(S, n, ck + (size_t)c * 7 * n, false, p->h0, st));
        const int64_t Ks = std::min<int64_t>(C, K - c * C);
        for (int64_t j = 0; j < Ks; j++)
            if ((rc = step(j, true))) return rc;
        for (int64_t j = Ks - 1; j >= 0; j--) {
            for (int sg = 3; sg >= 0; sg--) {
                const size_t k = (size_t)j * 4 + sg;
                CK(ctx, launch_adj_prop_in(n, P, sg, rec + k * n, A, gF, st));
                if (p->srp) {
                    ab.sun = rsun + k * 3 * n;
                    ab.dist = rdist + k * n;
                    rc = adj_enqueue(ctx, m, &p->eval, pl, n, ab.sun, ab.dist, ctx->arc_hits + k * n * R * nseg, ab,
                                     st, launches);
                    if (rc) return rc;
                    CK(ctx, launch_adj_sum(ge, n, m->h.n_mats, NP, acc, acc + NM2, st, true));
                    launches++;
                }
                CK(ctx, launch_adj_prop_out(n, P, sg, rec + k * n, A, gS, gD, st));
                launches += 2;
            }
            CK(ctx, launch_adj_prop_step(n, A, st));
            launches++;
        }
    }
    CK(ctx, launch_adj_prop_qsum(n, A, qsum, st));
    std::vector<PropAdj> ah(n);
    std::vector<double> accs((size_t)GE + 4);
    int flags = 0;
    CK(ctx, cudaMemcpyAsync(ah.data(), A, sizeof(PropAdj) * n, cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaMemcpyAsync(accs.data(), acc, sizeof(double) * (GE + 4), cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaMemcpyAsync(&flags, ctx->err_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaStreamSynchronize(st));
    std::vector<double> yo((size_t)6 * n), gy((size_t)6 * n);
    for (int i = 0; i < n; i++)
        for (int k = 0; k < 6; k++) {
            yo[6 * (size_t)i + k] = fin[i].y[k];
            gy[6 * (size_t)i + k] = ah[i].lam[k];
        }
    if (y1) CK(ctx, cudaMemcpy(y1, yo.data(), sizeof(double) * 6 * n, cudaMemcpyDefault));
    if (g_y0) CK(ctx, cudaMemcpy(g_y0, gy.data(), sizeof(double) * 6 * n, cudaMemcpyDefault));
    if (g_mat) CK(ctx, cudaMemcpy(g_mat, accs.data(), sizeof(double) * NM2, cudaMemcpyDefault));
    if (g_angle) CK(ctx, cudaMemcpy(g_angle, accs.data() + NM2, sizeof(double) * NP, cudaMemcpyDefault));
    if (g_q) CK(ctx, cudaMemcpy(g_q, accs.data() + GE, sizeof(double) * 4, cudaMemcpyDefault));
    if (stats)
        for (int i = 0; i < n; i++) {
            stats[i].steps = fin[i].steps;
            stats[i].rejects = fin[i].rejects;
            stats[i].evals = fin[i].evals;
            stats[i].t = fin[i].t;
            stats[i].status = fin[i].status;
            stats[i].reserved = 0;
            stats[i].h_next = fin[i].h;
        }
    ctx->last.launches = launches;
    ctx->last.trace_launches = trace_launches;
    if (flags & kFlagTimeout) return fail(ctx, SRP_ERR_TIMEOUT, "a work-queue wait gave up");
    if (flags & kFlagStack) return fail(ctx, SRP_ERR_STACK, "traversal stack bound reached");
    return SRP_OK;
}

srp_status srp_autotune(srp_ctx *ctx, int32_t mesh_id, const srp_eval_params *prm, int32_t *tile_w, double *ms)
{
    if (!ctx) return SRP_ERR_ARG;
    ctx->err.clear();
    Mesh *m = get_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, SRP_ERR_STATE, "bad mesh id %d", mesh_id);
    srp_status rc = check_eval_params(ctx, prm);
    if (rc) return rc;
    CK(ctx, cudaSetDevice(ctx->device));
    // 8 directions of a Fibonacci sphere, resident on the device
    const int nd = 8;
    std::vector<double> dirs(3 * nd);
    for (int i = 0; i < nd; i++) {
        double z = 1.0 - (2.0 * i + 1.0) / nd, r = std::sqrt(std::max(0.0, 1.0 - z * z));
        double ph = i * 3.14159265358979323846 * (3.0 - std::sqrt(5.0));
        dirs[3 * i] = r * std::cos(ph); dirs[3 * i + 1] = r * std::sin(ph); dirs[3 * i + 2] = z;
    }
    double *d = nullptr;
    CK(ctx, dalloc(&d, sizeof(double) * 9 * nd));
    struct Free { double *p; ~Free() { dfree(p); } } fr{d};
    CK(ctx, cudaMemcpy(d, dirs.data(), sizeof(double) * 3 * nd, cudaMemcpyHostToDevice));
    srp_eval_params q = *prm;
    q.flags = 0;
    const auto key = std::make_tuple((const void *)m, prm->N, prm->bounces + 1);
    const int cand[4] = {4, 8, 16, 32};
    double best = INFINITY;
    int best_w = 8;
    cudaEvent_t e0, e1;
    CK(ctx, cudaEventCreate(&e0));
    CK(ctx, cudaEventCreate(&e1));
    for (int c = 0; c < 4; c++) {
        ctx->tile_w[key] = cand[c];
        double tmin = INFINITY;
        for (int rep = 0; rep < 3; rep++) {
            CK(ctx, cudaEventRecord(e0, ctx->stream));
            rc = srp_eval_batch(ctx, mesh_id, &q, nd, d, nullptr, nullptr, d + 3 * nd, d + 6 * nd, nullptr);
            if (rc) break;
            CK(ctx, cudaEventRecord(e1, ctx->stream));
            CK(ctx, cudaEventSynchronize(e1));
            float t = 0.f;
            CK(ctx, cudaEventElapsedTime(&t, e0, e1));
            if (rep > 0) tmin = std::min(tmin, (double)t);  // the first run is a warm-up
        }
        if (rc) break;
        if (ms) ms[c] = tmin / nd;
        if (tmin < best) { best = tmin; best_w = cand[c]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tile_w[key] = best_w;
    if (rc) return rc;
    if (tile_w) *tile_w = best_w;
    return SRP_OK;
}

srp_status srp_set_tile_shape(srp_ctx *ctx, int32_t mesh_id, int32_t N, int32_t bounces, int32_t tile_w)
{
    if (!ctx) return SRP_ERR_ARG;
    ctx->err.clear();
    Mesh *m = get_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, SRP_ERR_ARG, "bad mesh id %d", mesh_id);
    if (tile_w != 4 && tile_w != 8 && tile_w != 16 && tile_w != 32) return fail(ctx, SRP_ERR_ARG, "tile width %d", tile_w);
    ctx->tile_w[std::make_tuple((const void *)m, N, bounces + 1)] = tile_w;
    return SRP_OK;
}

srp_status srp_propagate_batch(srp_ctx *ctx, const srp_prop_params *p, int32_t n, const srp_traj *tr, double *y1,
                               srp_prop_stats *stats)
{
    if (!ctx) return SRP_ERR_ARG;
    ctx->err.clear();
    if (!p || !tr || !y1 || n <= 0) return fail(ctx, SRP_ERR_ARG, "need params, n > 0 trajectories and y1");
    if (p->spad_table) return fail(ctx, SRP_ERR_ARG, "srp_propagate_batch takes no SPAD table");
    if (p->eval.n_diffuse != 0) return fail(ctx, SRP_ERR_ARG, "srp_propagate_batch takes no diffuse rays");
    if (p->method != SRP_RKF78 && p->method != SRP_RK4) return fail(ctx, SRP_ERR_ARG, "bad method");
    if (!(p->h0 > 0.0) || !(p->h_min >= 0.0) || p->max_steps <= 0) return fail(ctx, SRP_ERR_ARG, "bad step settings");
    if (p->method == SRP_RKF78 && (!(p->rtol > 0.0) || !(p->atol_pos > 0.0) || !(p->atol_vel > 0.0)))
        return fail(ctx, SRP_ERR_ARG, "tolerances must be > 0");
    if (!(p->eval.P0 >= 0.0) || !(p->eval.eps_rel >= 0.0)) return fail(ctx, SRP_ERR_ARG, "P0 and eps_rel must be >= 0");
    std::vector<Mesh *> mk(n);
    for (int i = 0; i < n; i++) {
        const srp_traj &t = tr[i];
        if (!(mk[i] = get_mesh(ctx, t.mesh_id))) return fail(ctx, SRP_ERR_STATE, "trajectory %d: bad mesh id", i);
        if (t.N < 1 || t.N > SRP_MAX_N || t.bounces < 0 || t.bounces > kMaxBounces || t.panel_mode < 0 ||
            t.panel_mode > 2 || (t.central != SRP_CENTRAL_EARTH && t.central != SRP_CENTRAL_SUN) ||
            (t.attitude != SRP_ATT_LVLH && t.attitude != SRP_ATT_INERTIAL))
            return fail(ctx, SRP_ERR_ARG, "trajectory %d: bad N, bounces, panel mode, central body or attitude", i);
        if (p->srp && !(mk[i]->mass > 0.0)) return fail(ctx, SRP_ERR_ARG, "trajectory %d: mesh mass must be > 0", i);
    }
    CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    memset(&ctx->last, 0, sizeof ctx->last);
    // trace tile shape per (mesh, N, bounces): tuned on request, else the context's choice
    std::vector<int> tw(n), tx(n), tiles(n);
    for (int i = 0; i < n; i++) {
        const auto key = std::make_tuple((const void *)mk[i], tr[i].N, tr[i].bounces + 1);
        if ((p->eval.flags & SRP_EVAL_AUTOTUNE) && !ctx->tile_w.count(key)) {
            srp_eval_params q{tr[i].N, tr[i].bounces, p->eval.P0, p->eval.eps_rel, tr[i].panel_mode, 0};
            srp_status rc = srp_autotune(ctx, tr[i].mesh_id, &q, nullptr, nullptr);
            if (rc) return rc;
        }
        tw[i] = tuned_tile_w(ctx, mk[i], tr[i].N, tr[i].bounces + 1);
        tile_grid(tr[i].N, tw[i], tx[i], tiles[i]);
    }
    // ---- device memory, owned by this call
    std::vector<void *> owned;
    struct Owner {
        std::vector<void *> &v;
        ~Owner() { for (void *q : v) dfree(q); }
    } owner{owned};
    int nbx = 0, max_verts = 0, max_dyn = 0;
    size_t n64 = 0, nview = 0, ntri = 0, nnode = 0;
    for (int i = 0; i < n; i++) {
        const MeshDev &h = mk[i]->h;
        nbx = std::max(nbx, tiles[i]);
        max_verts = std::max(max_verts, h.n_verts);
        max_dyn = std::max(max_dyn, h.n_dyn_tris);
        n64 += (size_t)h.n_dyn_verts * 3;
        nview += h.n_verts;
        ntri += (size_t)h.n_dyn_tris * 3;
        nnode += (size_t)h.n_dyn_nodes;
    }
    double *v64, *vv64, *io, *ang, *cfg;
    float4 *vview, *trec, *nodes;
    unsigned *cnt;
    float *rbox;
    SlotPose *pose;
    unsigned char *tctx;
    float *part;
    double *part1;
    unsigned *rticket;
    int *alist, *acount, *rbad;
    unsigned long long *pkey;
    unsigned *pcand, *bcount, *pcnt_blk;
    int4 *blist;
    int2 *btlist;
    SlotDesc *sd;
    PropState *S;
    size_t Rmax = 1;
    int max_tris = 0;
    for (int i = 0; i < n; i++) {
        Rmax = std::max(Rmax, (size_t)tr[i].N * tr[i].N);
        max_tris = std::max(max_tris, mk[i]->h.n_tris);
    }
    const bool raster = !(p->eval.flags & SRP_EVAL_TRAVERSE);
    const size_t bcap = std::min<size_t>((size_t)n * kBigPerSlot, (size_t)1 << 22);
    CK(ctx, dmalloc(owned, &v64, std::max<size_t>(n64, 1)));
    CK(ctx, dmalloc(owned, &vview, nview));
    CK(ctx, dmalloc(owned, &vv64, nview * 3));
    CK(ctx, dmalloc(owned, &trec, std::max<size_t>(ntri, 1)));
    CK(ctx, dmalloc(owned, &nodes, std::max<size_t>(nnode * kNode4, 1)));
    CK(ctx, dmalloc(owned, &cnt, std::max<size_t>(nnode, 1)));
    CK(ctx, dmalloc(owned, &rbox, (size_t)n * kMaxParts * 6));
    CK(ctx, dmalloc(owned, &io, (size_t)n * 18));
    CK(ctx, dmalloc(owned, &ang, (size_t)n * kMaxParts));
    CK(ctx, dmalloc(owned, &cfg, (size_t)n * 8));
    CK(ctx, dmalloc(owned, &pose, (size_t)n));
    CK(ctx, dmalloc(owned, &tctx, (size_t)n * trace_ctx_bytes()));
    CK(ctx, dmalloc(owned, &part, (size_t)n * nbx * 6));
    CK(ctx, dmalloc(owned, &pcnt_blk, (size_t)n * nbx * kCnt));
    CK(ctx, dmalloc(owned, &part1, (size_t)n * kRed1 * kPart));
    CK(ctx, dmalloc(owned, &rticket, (size_t)n));
    CK(ctx, dmalloc(owned, &alist, (size_t)n * nbx * kTileRays));
    CK(ctx, dmalloc(owned, &acount, (size_t)n * nbx));
    CK(ctx, dmalloc(owned, &sd, (size_t)n));
    CK(ctx, dmalloc(owned, &S, (size_t)n));
    CK(ctx, dmalloc(owned, &pkey, raster ? (size_t)n * Rmax : 1));
    CK(ctx, dmalloc(owned, &pcand, raster ? (size_t)n * Rmax * kPixCand : 1));
    CK(ctx, dmalloc(owned, &blist, raster ? bcap : 1));
    CK(ctx, dmalloc(owned, &btlist, raster ? bcap : 1));
    CK(ctx, dmalloc(owned, &bcount, 2));
    CK(ctx, dmalloc(owned, &rbad, (size_t)n));
    const bool queue = raster && (p->eval.flags & (SRP_EVAL_QUEUE | SRP_EVAL_TEST_WAIT_TIMEOUT));
    unsigned *qst = nullptr;
    CK(ctx, dmalloc(owned, &qst, queue ? qstate_words((size_t)n) : 1));
    CK(ctx, cudaMemsetAsync(bcount, 0, 2 * sizeof(unsigned), st));
    CK(ctx, cudaMemsetAsync(rbad, 0, sizeof(int) * n, st));
    double *d_sun = io, *d_dist = io + 3 * (size_t)n, *d_f = d_dist + n, *d_t = d_f + 3 * (size_t)n,
           *d_y0 = d_t + 3 * (size_t)n, *d_t01 = d_y0 + 6 * (size_t)n;
    CK(ctx, cudaMemsetAsync(cnt, 0, sizeof(unsigned) * std::max<size_t>(nnode, 1), st));
    CK(ctx, cudaMemsetAsync(rbox, 0, sizeof(float) * n * kMaxParts * 6, st));
    // per-trajectory slot storage, joint values and settings
    std::vector<SlotDesc> desc(n);
    std::vector<double> hang((size_t)n * kMaxParts, 0.0), hcfg((size_t)n * 8, 0.0), hy((size_t)n * 6), ht((size_t)n * 2);
    size_t o64 = 0, oview = 0, otri = 0, onode = 0;
    for (int i = 0; i < n; i++) {
        const Mesh *m = mk[i];
        const MeshDev &h = m->h;
        SlotDesc &d = desc[i];
        d.mesh = m->d;
        d.sb.vert64 = v64 + o64;
        d.sb.vview = vview + oview;
        d.sb.vview64 = vv64 + oview * 3;
        d.sb.tri = trec + otri;
        d.sb.node = nodes + onode * kNode4;
        d.sb.counter = cnt + onode;
        d.sb.root_box = rbox + (size_t)i * kMaxParts * 6;
        if (h.n_dyn_nodes > 0)
            CK(ctx, cudaMemcpyAsync(d.sb.node, m->node_tmpl_dyn, sizeof(float4) * kNode4 * h.n_dyn_nodes,
                                    cudaMemcpyDeviceToDevice, st));
        o64 += (size_t)h.n_dyn_verts * 3;
        oview += h.n_verts;
        otri += (size_t)h.n_dyn_tris * 3;
        onode += h.n_dyn_nodes;
        if (tr[i].angles) {
            for (int k = 0; k < h.n_parts; k++) hang[(size_t)i * kMaxParts + k] = tr[i].angles[k];
            d.angles = ang + (size_t)i * kMaxParts;
        } else {
            d.angles = m->angles_d;
        }
        d.N = tr[i].N;
        d.nseg = tr[i].bounces + 1;
        d.panel_mode = tr[i].panel_mode;
        d.tile_w = tw[i];
        d.tiles_x = tx[i];
        d.tiles = tiles[i];
        double *c = &hcfg[8 * (size_t)i];
        c[0] = tr[i].central;
        c[1] = tr[i].attitude;
        for (int k = 0; k < 4; k++) c[2 + k] = tr[i].q[k];
        c[6] = m->mass;
        for (int k = 0; k < 6; k++) hy[6 * (size_t)i + k] = tr[i].y0[k];
        ht[2 * (size_t)i] = tr[i].t0;
        ht[2 * (size_t)i + 1] = tr[i].t1;
    }
    CK(ctx, cudaMemcpyAsync(ang, hang.data(), sizeof(double) * hang.size(), cudaMemcpyHostToDevice, st));
    CK(ctx, cudaMemcpyAsync(cfg, hcfg.data(), sizeof(double) * hcfg.size(), cudaMemcpyHostToDevice, st));
    CK(ctx, cudaMemcpyAsync(d_y0, hy.data(), sizeof(double) * hy.size(), cudaMemcpyHostToDevice, st));
    CK(ctx, cudaMemcpyAsync(d_t01, ht.data(), sizeof(double) * ht.size(), cudaMemcpyHostToDevice, st));
    CK(ctx, cudaMemsetAsync(ctx->err_flags, 0, sizeof(int), st));
    CK(ctx, cudaMemsetAsync(ctx->stats, 0, 16 * sizeof(unsigned long long), st));
    CK(ctx, cudaMemsetAsync(ctx->prop_done, 0, sizeof(int), st));
    PropDev P{};
    P.method = p->method; P.j2 = p->j2; P.sun3 = p->sun3; P.srp = p->srp;
    P.epoch_mjd_tt = p->epoch_mjd_tt;
    P.rtol = p->rtol; P.atol_pos = p->atol_pos; P.atol_vel = p->atol_vel;
    P.h0 = p->h0; P.h_min = p->h_min; P.h_max = p->h_max; P.max_steps = p->max_steps;
    CK(ctx, launch_prop_init(S, n, d_y0, d_t01, P, cfg, ctx->prop_done, st));
    const int nstage = p->method == SRP_RK4 ? 4 : 13;
    // slot k runs trajectory act[k]; finished ones leave through compaction
    std::vector<int> act(n);
    for (int i = 0; i < n; i++) act[i] = i;
    std::vector<PropState> fin(n), peek(n);
    std::vector<char> have(n, 0);
    cudaGraphExec_t exec = nullptr;
    struct GraphGuard {
        cudaGraphExec_t &e;
        ~GraphGuard() { if (e) cudaGraphExecDestroy(e); }
    } gg{exec};
    int64_t launches = 0, trace_launches = 0, graphs = 0;
    auto capture = [&](int na) -> srp_status {
        // descriptors of the running trajectories, their tiles laid end to end
        std::vector<SlotDesc> dd(na);
        int t0 = 0, r0 = 0, mv = 0, md = 0, mp = 0, ms = 0;
        for (int k = 0; k < na; k++) {
            dd[k] = desc[act[k]];
            mp = std::max(mp, mk[act[k]]->h.n_parts);
            ms = std::max(ms, dd[k].nseg);
            dd[k].tile0 = t0;
            t0 += trace_blocks(dd[k].tiles);
            dd[k].rast0 = r0;
            r0 += (mk[act[k]]->h.n_tris + 127) / 128;
            mv = std::max(mv, mk[act[k]]->h.n_verts);
            md = std::max(md, mk[act[k]]->h.n_dyn_tris);
        }
        CK(ctx, cudaMemcpyAsync(sd, dd.data(), sizeof(SlotDesc) * na, cudaMemcpyHostToDevice, st));
        CK(ctx, cudaStreamSynchronize(st));
        TraceArgs a{};
        a.sd = sd;
        a.n_slots = na;
        a.n_tiles = t0;
        a.pose = pose;
        a.tctx = tctx;
        a.eps_rel = p->eval.eps_rel;
        a.n_blocks_x = nbx;
        a.partials = part;
        a.pcounts = pcnt_blk;
        a.partials1 = part1;
        a.red_ticket = rticket;
        a.ctx_parts = mp;
        a.hpt_segs = ms;
        a.amb_list = alist;
        a.amb_count = acount;
        a.ray_stride = Rmax;
        if (raster) {
            a.raster = 1;
            a.rast_tris = max_tris;
            a.pix_key = pkey;
            a.pix_cand = pcand;
            a.big = blist;
            a.big_cap = (int)bcap;
            a.big_count = bcount;
            a.bigt = btlist;
            a.bigt_count = bcount + 1;
            a.rast_bad = rbad;
            if (queue) {
                a.queue = 1;
                a.wait_test = (p->eval.flags & SRP_EVAL_TEST_WAIT_TIMEOUT) ? 1 : 0;
                a.n_small_items = r0;
                a.qstate = qst;
            }
        }
        cudaGraph_t graph = nullptr;
        CK(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        // without ray tracing a stage's acceleration and the next stage share no
        // launch; with it, a step starts from its first stage's state, made by the
        // previous step's last launch or by the launch after this capture
        for (int sg = 0; sg < nstage && e == cudaSuccess; sg++) {
            if (!p->srp) e = launch_prop_stage(S, na, P, sg, d_sun, d_dist, st);
            if (p->srp) {
                if (e == cudaSuccess) e = launch_pose(sd, d_sun, d_dist, p->eval.P0, 0, na, pose, st);
                if (e == cudaSuccess) e = launch_vertices(sd, pose, na, mv, st);
                // the refit beside frame and raster, joined before the trace
                if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_refit_fork[0], st);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->aux[0], ctx->ev_refit_fork[0], 0);
                if (e == cudaSuccess) e = launch_refit(sd, pose, na, md, ctx->aux[0]);
                if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_refit_join[0], ctx->aux[0]);
                if (e == cudaSuccess) e = launch_frame(a, na, st);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->ev_refit_join[0], 0);
                if (e == cudaSuccess) e = launch_trace(a, na, st);
                if (e == cudaSuccess) e = launch_reduce(a, na, 0, d_f, d_t, ctx->err_flags, nullptr, st);
                if (e == cudaSuccess) e = launch_prop_next(S, na, P, sg, d_f, d_sun, d_dist, ctx->prop_done, nullptr, 0, st);
            } else if (e == cudaSuccess) {
                e = launch_prop_accel(S, na, P, sg, d_f, st);
            }
        }
        if (e == cudaSuccess && !p->srp) e = launch_prop_control(S, na, P, ctx->prop_done, nullptr, 0, st);
        cudaError_t ce = cudaStreamEndCapture(st, &graph);
        if (e != cudaSuccess || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return fail(ctx, SRP_ERR_CUDA, "batch step capture failed: %s",
                        cudaGetErrorString(e != cudaSuccess ? e : ce));
        }
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return fail(ctx, SRP_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
        graphs++;
        // the first stage of the running trajectories' next step, in their (new) slots
        if (p->srp) CK(ctx, launch_prop_stage(S, na, P, 0, d_sun, d_dist, st));
        return SRP_OK;
    };
    int na = n;
    srp_status rc = capture(na);
    if (rc) return rc;
    const int poll_max = p->poll > 0 ? p->poll : 16;
    // per stage with the SRP: pose, vertices, refit, frame, the raster launches,
    // trace, the reduction, then the acceleration with
    // the next stage (control at the last); without it stage, acceleration, and control
    const int per_step = p->srp ? nstage * (1 + 6 + (raster ? raster_launches(n, queue) : 0)) : nstage * 2 + 1;
    for (int64_t round = 0; round < p->max_steps + 2 && na > 0; round++) {
        int done = 0;
        CK(ctx, cudaMemcpyAsync(&done, ctx->prop_done, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(ctx, cudaMemcpyAsync(peek.data(), S, sizeof(PropState) * na, cudaMemcpyDeviceToHost, st));
        CK(ctx, cudaStreamSynchronize(st));
        if (done >= na) break;
        if (na >= 4 && 2 * done >= na) {
            // compaction: keep the running trajectories in the first slots
            std::vector<int> keep;
            std::vector<PropState> ks;
            for (int k = 0; k < na; k++) {
                if (peek[k].done) { fin[act[k]] = peek[k]; have[act[k]] = 1; }
                else { keep.push_back(act[k]); ks.push_back(peek[k]); }
            }
            act = keep;
            na = (int)act.size();
            CK(ctx, cudaMemcpyAsync(S, ks.data(), sizeof(PropState) * na, cudaMemcpyHostToDevice, st));
            CK(ctx, cudaMemsetAsync(ctx->prop_done, 0, sizeof(int), st));
            if ((rc = capture(na))) return rc;
            continue;
        }
        double need = 1.0;
        for (int k = 0; k < na; k++) {
            const PropState &X = peek[k];
            if (X.done) continue;
            need = std::max(need, (X.t1 - X.t) / std::max(X.h, 1e-300));
        }
        const int launch = (int)std::min<double>(poll_max, std::max(1.0, std::ceil(need)));
        for (int k = 0; k < launch; k++) CK(ctx, cudaGraphLaunch(exec, st));
        launches += (int64_t)launch * per_step;
        trace_launches += (int64_t)launch * nstage;
    }
    if (na > 0) {
        CK(ctx, cudaMemcpyAsync(peek.data(), S, sizeof(PropState) * na, cudaMemcpyDeviceToHost, st));
        CK(ctx, cudaStreamSynchronize(st));
        for (int k = 0; k < na; k++) { fin[act[k]] = peek[k]; have[act[k]] = 1; }
    }
    int flags = 0;
    CK(ctx, cudaMemcpy(&flags, ctx->err_flags, sizeof(int), cudaMemcpyDeviceToHost));
    std::vector<double> yo((size_t)6 * n);
    srp_status out = SRP_OK;
    for (int i = 0; i < n; i++) {
        for (int k = 0; k < 6; k++) yo[6 * (size_t)i + k] = fin[i].y[k];
        if (stats) {
            stats[i].steps = fin[i].steps;
            stats[i].rejects = fin[i].rejects;
            stats[i].evals = fin[i].evals;
            stats[i].t = fin[i].t;
            stats[i].status = fin[i].status;
            stats[i].reserved = 0;
        }
        if (!have[i] || fin[i].status || !fin[i].done) out = SRP_ERR_STEP;
    }
    CK(ctx, cudaMemcpy(y1, yo.data(), sizeof(double) * 6 * n, cudaMemcpyDefault));
    ctx->last.launches = launches;
    ctx->last.trace_launches = trace_launches;
    if (flags & kFlagTimeout) return fail(ctx, SRP_ERR_TIMEOUT, "a work-queue wait gave up");
    if (flags & kFlagStack) return fail(ctx, SRP_ERR_STACK, "traversal stack bound reached");
    if (out) return fail(ctx, SRP_ERR_STEP, "a trajectory hit h_min or max_steps");
    (void)graphs;
    return SRP_OK;
}

}  // extern "C"
