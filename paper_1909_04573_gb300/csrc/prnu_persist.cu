// prnu_persist.cu -- host side of the persistent multi-camera pipeline
// (k_persist.cu): the work-queue planner, the workspace layout and the entry
// points prnu_workspace_size_persistent, prnu_fingerprint_accumulate_persistent,
// prnu_persistent_status and prnu_persistent_wait_probe.
#include <algorithm>
#include <cstring>
#include <vector>

#include "abi_internal.cuh"

using namespace prnu;
using namespace prnu::abi;

namespace {

constexpr double kDefaultBudgetMs = 2000.0;

struct Plan {
    std::vector<PGroup> groups;
    std::vector<PCam> cams;
    std::vector<PGeo> geos;
    std::vector<PSeg> segs;
    int L = 0, NS = 0, nslots = 0, total = 0;
    size_t slot_bytes = 0;
    // workspace offsets
    size_t done = 0, blob = 0, g_off = 0, c_off = 0, geo_off = 0, seg_off = 0, slots = 0, end = 0;
    std::vector<unsigned char> bytes;  // groups | cams | geos | segs, copied to ws + blob
};

int sda_seg(int C) { return C == 3 ? 1024 : 4096; }
int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

PGeo make_geo(int H, int W, int C, int L) {
    PGeo g;
    std::memset(&g, 0, sizeof g);
    g.H = H;
    g.W = W;
    g.C = C;
    g.Hp = padded(H, L);
    g.Wp = padded(W, L);
    const Layout lo = make_layout(H, W, C, L, true, SB_F32);
    g.X = (long long)lo.X;
    for (int l = 0; l <= kMaxLevels; ++l) {
        g.LLh[l] = (long long)lo.LLh[l];
        g.LLl[l] = (long long)lo.LLl[l];
        g.Rn[l] = (long long)lo.Rn[l];
        g.D[l] = (long long)lo.D[l];
        g.N[l] = (long long)lo.N[l];
    }
    // items per stage: tiles (the same tilings as the device decode in
    // k_persist.cu) grouped kPTiles* to an item
    g.cnt[0] = cdiv((long long)H * cdiv(W, sda_seg(C)), kPTilesSda);
    for (int l = 1; l <= L; ++l) {
        g.cnt[l] = cdiv((long long)C * cdiv(g.Hp >> l, 16) * cdiv(g.Wp >> l, 32), kPTilesAna);  // 16 x 32 outputs
        g.cnt[L + l] = cdiv(3LL * C * cdiv(g.Hp >> l, 32) * cdiv(g.Wp >> l, 32), kPTilesShr);   // 32 x 32
    }
    for (int l = L; l >= 2; --l)
        g.cnt[3 * L + 1 - l] = cdiv((long long)C * cdiv(g.Hp >> (l - 1), 32) * cdiv(g.Wp >> (l - 1), 32), kPTilesSyn);
    g.cnt[3 * L] = cdiv((long long)C * cdiv(H, 32) * cdiv(W, 32), kPTilesFin);  // level-1 synthesis + MLE
    return g;
}

// Host copy of the device's dependency rule (deps_of in k_persist.cu):
// (group, stage) pairs whose every item must precede an item of (g, s).
int host_deps(const Plan &p, int g, int s, int out[3][2]) {
    const int L = p.L;
    int n = 0;
    auto add = [&](int dg, int ds) {
        out[n][0] = dg;
        out[n][1] = ds;
        ++n;
    };
    if (s == 0) {
        if (g >= p.nslots) add(g - p.nslots, 3 * L);
    } else if (s <= L) {
        add(g, s - 1);
    } else if (s <= 2 * L) {
        add(g, s - L);
    } else if (s < 3 * L) {
        const int l = 3 * L + 1 - s;
        add(g, L + l);
        if (l < L) add(g, s - 1);
    } else {
        add(g, L + 1);
        if (L >= 2) add(g, 3 * L - 1);
        if (p.groups[g].prev >= 0) add(p.groups[g].prev, 3 * L);
    }
    return n;
}

struct Chunk {
    int group, stage, first, count;
};

// The queue: in wave w, the SDA sums of group w, the analysis and shrink of
// group w-1 and the synthesis and MLE step of group w-2, each stage cut into
// chunks and the three lists interleaved in proportion to their item counts.
// Every chunk is checked to come after all items of the stages it depends on.
prnu_status build_queue(Plan &p) {
    const int G = (int)p.groups.size(), L = p.L;
    std::vector<int> emitted((size_t)G * p.NS, 0);
    auto cnt = [&](int g, int s) { return p.geos[p.groups[g].geo].cnt[s]; };
    auto chunks_of = [&](int g, const std::vector<int> &stages, std::vector<Chunk> &out) {
        for (int s : stages) {
            const int n = cnt(g, s);
            const int ch = std::max(256, (n + 7) / 8);
            for (int f = 0; f < n; f += ch) out.push_back(Chunk{g, s, f, std::min(ch, n - f)});
        }
    };
    std::vector<int> front, back;
    for (int l = 1; l <= L; ++l) {
        front.push_back(l);
        front.push_back(L + l);
    }
    for (int l = L; l >= 2; --l) back.push_back(3 * L + 1 - l);
    back.push_back(3 * L);
    int total = 0;
    for (int w = 0; w < G + 2; ++w) {
        std::vector<Chunk> lists[3];
        if (w < G) chunks_of(w, {0}, lists[0]);
        if (w - 1 >= 0 && w - 1 < G) chunks_of(w - 1, front, lists[1]);
        if (w - 2 >= 0 && w - 2 < G) chunks_of(w - 2, back, lists[2]);
        long long tot[3] = {0, 0, 0}, done[3] = {0, 0, 0};
        size_t pos[3] = {0, 0, 0};
        for (int k = 0; k < 3; ++k)
            for (auto &c : lists[k]) tot[k] += c.count;
        for (;;) {
            int pick = -1;
            double best = 2.0;
            for (int k = 0; k < 3; ++k) {
                if (pos[k] >= lists[k].size()) continue;
                const double r = (double)done[k] / (double)tot[k];
                if (r < best) {
                    best = r;
                    pick = k;
                }
            }
            if (pick < 0) break;
            const Chunk c = lists[pick][pos[pick]++];
            done[pick] += c.count;
            int dep[3][2];
            const int nd = host_deps(p, c.group, c.stage, dep);
            for (int i = 0; i < nd; ++i)
                if (emitted[(size_t)dep[i][0] * p.NS + dep[i][1]] != cnt(dep[i][0], dep[i][1]))
                    return fail(PRNU_EINVAL, "internal: work queue order (group %d stage %d before group %d stage %d)",
                                c.group, c.stage, dep[i][0], dep[i][1]);
            p.segs.push_back(PSeg{total, c.group, c.stage, c.first});
            emitted[(size_t)c.group * p.NS + c.stage] += c.count;
            total += c.count;
        }
    }
    p.total = total;
    return PRNU_OK;
}

// Tables and workspace layout (no device work).
void finish_layout(Plan &p) {
    const size_t G = p.groups.size();
    size_t off = align_up(sizeof(PHeader), kAlign);
    p.done = off;
    off = align_up(off + G * p.NS * sizeof(int), kAlign);
    p.blob = off;
    size_t b = 0;
    auto put = [&](const void *src, size_t n) {
        const size_t o = b;
        p.bytes.resize(o + align_up(n, 16));
        if (n) std::memcpy(p.bytes.data() + o, src, n);
        b = p.bytes.size();
        return p.blob + o;
    };
    p.bytes.clear();
    p.g_off = put(p.groups.data(), G * sizeof(PGroup));
    p.c_off = put(p.cams.data(), p.cams.size() * sizeof(PCam));
    p.geo_off = put(p.geos.data(), p.geos.size() * sizeof(PGeo));
    p.seg_off = put(p.segs.data(), p.segs.size() * sizeof(PSeg));
    off = align_up(p.blob + b, kAlign);
    p.slots = off;
    p.end = off + (size_t)p.nslots * p.slot_bytes;
}

prnu_status plan_cameras(const prnu_camera *cams, int ncams, const prnu_params *params, int slots, Plan &p) {
    if (!cams || ncams < 1) return fail(PRNU_EINVAL, "cams is NULL or ncams < 1");
    if (slots < 3 || slots > 64) return fail(PRNU_EINVAL, "slots must be in [3, 64] (got %d)", slots);
    prnu_status s;
    for (int i = 0; i < ncams; ++i) {
        const prnu_camera &c = cams[i];
        if ((s = check_geometry(c.H, c.W, c.C)) != PRNU_OK) return s;
        if ((s = check_params(params, c.H, c.W, nullptr)) != PRNU_OK) return s;
        if (!c.num || !c.den) return fail(PRNU_EINVAL, "camera %d: num/den is NULL", i);
        if ((s = check_frames(c.frames, c.m, c.H, c.W, c.C, c.frame_stride, c.row_pitch, c.d, 1)) != PRNU_OK)
            return s;
    }
    if (params->dtype != PRNU_DTYPE_F32 || params->frame_dtype != PRNU_FRAMES_U8)
        return fail(PRNU_EUNSUPPORTED, "the persistent pipeline takes uint8 frames and float32 subbands");
    p.L = params->levels;
    p.NS = 3 * p.L + 1;
    p.nslots = slots;
    for (int i = 0; i < ncams; ++i) {
        const prnu_camera &c = cams[i];
        int geo = -1;
        for (size_t k = 0; k < p.geos.size(); ++k)
            if (p.geos[k].H == c.H && p.geos[k].W == c.W && p.geos[k].C == c.C) geo = (int)k;
        if (geo < 0) {
            if ((int)p.geos.size() == kPMaxGeos)
                return fail(PRNU_EINVAL, "at most %d distinct geometries per call", kPMaxGeos);
            geo = (int)p.geos.size();
            p.geos.push_back(make_geo(c.H, c.W, c.C, p.L));
            p.slot_bytes = std::max(p.slot_bytes, align_up(make_layout(c.H, c.W, c.C, p.L, true, SB_F32).end, kAlign));
        }
        p.cams.push_back(PCam{c.num, c.den});
        const int ng = (c.m + c.d - 1) / c.d;
        int prev = -1;
        for (int k = 0; k < ng; ++k) {
            const int j0 = k * c.d, j1 = std::min(c.m, j0 + c.d);
            PGroup g;
            g.frames = c.frames + (size_t)j0 * c.frame_stride;
            g.frame_stride = (long long)c.frame_stride;
            g.row_pitch = (long long)c.row_pitch;
            g.n = j1 - j0;
            g.cam = i;
            g.geo = geo;
            g.prev = prev;
            prev = (int)p.groups.size();
            p.groups.push_back(g);
        }
    }
    for (int i = 0; i < ncams; ++i)
        for (int j = 0; j < i; ++j)
            if (cams[i].num == cams[j].num || cams[i].den == cams[j].den)
                return fail(PRNU_EINVAL, "cameras %d and %d share num/den", j, i);
    if ((s = build_queue(p)) != PRNU_OK) return s;
    finish_layout(p);
    return PRNU_OK;
}

prnu_status launch_plan(prnu_ctx *ctx, Plan &p, const prnu_params *params, const Win &win, double budget_ms,
                        char *ws, cudaStream_t st) {
    CU(cudaMemsetAsync(ws, 0, p.blob, st));  // header and completion counts
    CU(launch_put_bytes(p.bytes.data(), p.bytes.size(), ws + p.blob, st));
    PArgs a;
    std::memset(&a, 0, sizeof a);
    a.hdr = reinterpret_cast<PHeader *>(ws);
    a.groups = reinterpret_cast<const PGroup *>(ws + p.g_off);
    a.cams = reinterpret_cast<const PCam *>(ws + p.c_off);
    a.geos = reinterpret_cast<const PGeo *>(ws + p.geo_off);
    a.segs = reinterpret_cast<const PSeg *>(ws + p.seg_off);
    a.done = reinterpret_cast<int *>(ws + p.done);
    a.slots = ws + p.slots;
    a.slot_bytes = (long long)p.slot_bytes;
    a.nslots = p.nslots;
    a.L = p.L;
    a.NS = p.NS;
    a.nseg = (int)p.segs.size();
    a.total = p.total;
    a.G = (int)p.groups.size();
    a.s2 = params ? params->sigma0 * params->sigma0 : 0.f;
    a.win = win;
    a.f = ctx->filt;
    a.budget_ns = (long long)((budget_ms > 0.0 ? budget_ms : kDefaultBudgetMs) * 1e6);
    const bool comp = params && params->compensated;
    const bool std4 = win.n == 4 && win.r[0] == 1 && win.r[1] == 2 && win.r[2] == 3 && win.r[3] == 4;
    const long long blocks = std::min<long long>((long long)ctx->sms * persist_blocks_per_sm(comp, std4),
                                                 std::max(p.total, 1));
    double fr = 0.0;
    for (const PGroup &g : p.groups) {
        const PGeo &ge = p.geos[g.geo];
        fr += (double)g.n * ge.H * ge.W * ge.C;
    }
    Launch t(ctx, "persist", st, 1, fr);
    CU(launch_persist(a, comp, std4, (int)blocks, st));
    return PRNU_OK;
}

}  // namespace

extern "C" {

prnu_status prnu_workspace_size_persistent(prnu_ctx *ctx, const prnu_camera *cams, int ncams,
                                           const prnu_params *params, int slots, size_t *bytes) {
    if (!ctx || !bytes) return fail(PRNU_EINVAL, "ctx/bytes is NULL");
    Plan p;
    prnu_status s = plan_cameras(cams, ncams, params, slots, p);
    if (s != PRNU_OK) return s;
    *bytes = p.end;
    return PRNU_OK;
}

prnu_status prnu_fingerprint_accumulate_persistent(prnu_ctx *ctx, const prnu_camera *cams, int ncams,
                                                   const prnu_params *params, int slots, double wait_budget_ms,
                                                   void *ws, size_t ws_bytes, void *stream) {
    if (!ctx) return fail(PRNU_EINVAL, "ctx is NULL");
    if (!(wait_budget_ms >= 0.0) || wait_budget_ms > 6e5) return fail(PRNU_EINVAL, "wait_budget_ms must be in [0, 6e5]");
    Plan p;
    prnu_status s = plan_cameras(cams, ncams, params, slots, p);
    if (s != PRNU_OK) return s;
    Win win;
    if ((s = check_params(params, cams[0].H, cams[0].W, &win)) != PRNU_OK) return s;
    if ((s = check_ws(ws, ws_bytes, p.end)) != PRNU_OK) return s;
    DeviceGuard g(ctx->device);
    return launch_plan(ctx, p, params, win, wait_budget_ms, static_cast<char *>(ws), S(stream));
}

prnu_status prnu_persistent_status(prnu_ctx *ctx, const void *ws, size_t ws_bytes, void *stream, int *fail_info) {
    if (!ctx || !ws) return fail(PRNU_EINVAL, "ctx/ws is NULL");
    if (ws_bytes < sizeof(PHeader)) return fail(PRNU_EINVAL, "workspace smaller than the queue header");
    DeviceGuard g(ctx->device);
    PHeader h;
    CU(cudaMemcpyAsync(&h, ws, sizeof h, cudaMemcpyDeviceToHost, S(stream)));
    CU(cudaStreamSynchronize(S(stream)));
    if (fail_info) {
        fail_info[0] = h.fail_item;
        fail_info[1] = h.fail_group;
        fail_info[2] = h.fail_stage;
    }
    if (h.status == PRNU_ETIMEOUT)
        return fail(PRNU_ETIMEOUT,
                    "a bounded wait of the persistent pipeline gave up: item %d (group %d, stage %d); %d block(s) "
                    "timed out",
                    h.fail_item, h.fail_group, h.fail_stage, h.fail_blocks);
    if (h.status != 0) return fail(PRNU_ECUDA, "persistent pipeline status %d", h.status);
    return PRNU_OK;
}

prnu_status prnu_persistent_wait_probe(prnu_ctx *ctx, double wait_budget_ms, void *ws, size_t ws_bytes, void *stream) {
    if (!ctx) return fail(PRNU_EINVAL, "ctx is NULL");
    if (!(wait_budget_ms > 0.0) || wait_budget_ms > 1e4) return fail(PRNU_EINVAL, "wait_budget_ms must be in (0, 1e4]");
    Plan p;
    p.L = 1;
    p.NS = 4;
    p.nslots = 3;
    PGroup g;
    std::memset(&g, 0, sizeof g);
    g.prev = -1;
    p.groups.push_back(g);
    p.geos.push_back(make_geo(16, 16, 1, 1));
    p.segs.push_back(PSeg{0, 0, kPProbeStage, 0});
    p.total = 1;
    p.slot_bytes = 0;
    finish_layout(p);
    prnu_status s;
    if ((s = check_ws(ws, ws_bytes, p.end)) != PRNU_OK) return s;
    Win win;
    std::memset(&win, 0, sizeof win);
    DeviceGuard dg(ctx->device);
    return launch_plan(ctx, p, nullptr, win, wait_budget_ms, static_cast<char *>(ws), S(stream));
}

}  // extern "C"
