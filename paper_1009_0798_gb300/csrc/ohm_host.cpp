// ohm_host.cpp -- hierarchy construction, device memory plan, multigrid schedule and the
// C ABI of libohm (declared in include/ohm.h).  Every arithmetic step runs in the kernels of
// ohm_kernels.cu; this file only builds index tables, allocates once and enqueues launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "ohm.h"
#include "ohm_internal.h"

using namespace ohm;

namespace {

constexpr int MAX_LEVELS = 8;
// lexicographic grids of more cells than this are stepped by grid-wide launches; the rest, down
// to the coarsest, by the one-block solver (k_bottom: one thread block per instance)
constexpr int MAX_BOTTOM_CELLS = 16384;
// mixed precision: coarse grids of at most this many cells (16^3), with power-of-two extents, are
// not blocked; the coarsest-grid solver runs them in shared memory
constexpr int64_t MIN_BLOCKED_CELLS = 4096;

inline int wrapi(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}
inline int64_t key3(int i, int j, int k) { return ((int64_t)k << 42) | ((int64_t)j << 21) | (int64_t)i; }

uint64_t morton(int i, int j, int k) {
    uint64_t m = 0;
    for (int b = 0; b < 21; b++)
        m |= ((uint64_t)((i >> b) & 1) << (3 * b)) | ((uint64_t)((j >> b) & 1) << (3 * b + 1)) |
             ((uint64_t)((k >> b) & 1) << (3 * b + 2));
    return m;
}

// Host tables of one blocked grid; `dev` receives the device pointers after upload.
struct HGrid {
    int level = 0;              // AMR level, or -1 for a base multigrid grid
    int dims[3] = {0, 0, 0};    // cells
    int nb[3] = {0, 0, 0};      // blocks per axis
    double h = 0;
    int off = 0;                // first block in the caller's arrays (AMR levels)
    std::vector<int> bijk;      // 3 per block
    std::unordered_map<int64_t, int> index;
    std::vector<int> nbr, parent, child, origin, freg, rsrc, gslot, slot_block;
    std::vector<uint8_t> covered, octant;
    int slot0 = 0, nslot = 0;
    int inst_nblk = 0;          // batches: blocks per instance
    bool brick = false;         // blocks pair up as x-neighbours (2q, 2q+1), every neighbour present
    bool octet = false;         // the children of coarser-grid block c are blocks 8c .. 8c+7
    GridDev dev;
    int find(int i, int j, int k) const {
        auto it = index.find(key3(wrapi(i, nb[0]), wrapi(j, nb[1]), wrapi(k, nb[2])));
        return it == index.end() ? -1 : it->second;
    }
    int n() const { return (int)(bijk.size() / 3); }
};

struct Buffers {  // precision-dependent multigrid arrays (element type T)
    void *r = nullptr, *e = nullptr, *e2 = nullptr, *eta = nullptr, *inv = nullptr;
};

}  // namespace

struct ohm_hier {
    ohm_hier_desc d{};
    cudaStream_t s = nullptr;
    bool mixed = false;
    bool ff = false;     // OHM_MIXED_FF: float-float outer residual, S in float-float form
    int nlev = 0;
    int64_t nblocks = 0;
    std::vector<int32_t> lijk;
    std::vector<HGrid> amr;       // AMR levels
    std::vector<HGrid> mg;        // blocked base multigrid grids m = 1 .. (index m-1)
    std::vector<std::array<int, 3>> small;  // lexicographic grids below the last blocked one
    int nslot = 0, nreg = 0, nrsrc = 0;
    std::vector<int> rsrc_tab;

    // device memory (one pool)
    void *pool = nullptr;
    double *S = nullptr, *eta64 = nullptr, *Bscr = nullptr, *ghostB = nullptr, *ghostEta64 = nullptr;
    double *reg = nullptr, *partials = nullptr, *dnorm = nullptr, *redscr = nullptr;
    int *d_rsrc = nullptr, *d_err = nullptr;
    void *ghostE = nullptr, *ghostEtaT = nullptr;
    void *rout = nullptr, *eacc = nullptr;  // mixed precision: float32 outer residual, inner correction
    // FGMRES inner solve (mixed precision, krylov > 0): Arnoldi basis, preconditioned vectors,
    // per-block inner-product weights, multi-dot scratch and results (device and pinned host)
    float *kv[KMAX + 1] = {}, *kz[KMAX] = {};
    double *wblk = nullptr, *kpart = nullptr, *kdots = nullptr, *hdots = nullptr;
    // batched FGMRES: per-instance coefficients (device) and the instance of every block
    float *kcoef = nullptr;
    int *binst = nullptr;
    std::vector<double> wblk_host;
    Buffers amrbuf;               // AMR levels, all blocks
    std::vector<Buffers> mgbuf;   // blocked multigrid grids
    Buffers smallbuf[MAX_SMALL];  // small grids (t stored in e2)
    double *hnorm = nullptr;      // pinned host copy: 4 doubles + error word
    int *flag_dev = nullptr;      // device address of the eta-comparison flag in hnorm (mapped)
    double *hnorm_dev = nullptr;  // device address of hnorm itself (mapped), null if not mapped

    bool ff_mid = false;          // OHM_MIXED_FF_CHECKED: intermediate outer residuals in float-float
    bool inv_all = false;         // the inverse diagonals of every grid are those of inv_dt
    bool eta_set = false;
    double inv_dt = NAN;
    bool has_S = false;
    double last_dt = 0;

    // batches (n_instances >= 1): K instances of one block structure, stacked level by level
    bool batched = false;
    int K = 1;
    int64_t nblk_inst = 0;        // blocks of one instance
    double *eta_user = nullptr;   // eta as set (the operator uses eta * dt per instance)
    double *bscale = nullptr;     // per-block eta scale (the instance's dt)
    double *dnormK = nullptr;     // [K][4] per-instance norm sums
    double *hnormK = nullptr;     // pinned copy
    uint8_t *imask_d = nullptr, *imask_h = nullptr;  // per-instance update mask (device, pinned)
    std::vector<double> cur_scale;
    bool eta_dirty = false;
    InstRanges ranges;
    int smoother = 0;             // 0: fused red+black sweep where possible, 1: two colour passes
    const uint8_t *cmask = nullptr;  // compute mask of batched iterations (null: every instance)
    double active_frac = 1.0;        // share of instances the compute mask lets through (timing)
    // CUDA graph of the batched inner iteration
    cudaGraphExec_t graph = nullptr;
    bool graph_warm = false, graph_failed = false;
    int64_t graph_launches = 0;
    // batched FGMRES: per-instance scalars on the device, a pinned staging area (target, cycles,
    // run and live flags) and the CUDA graph of one restart cycle
    FgState fg;
    char *fg_host = nullptr;
    cudaGraphExec_t fg_graph = nullptr;
    bool fg_warm = false, fg_failed = false;
    int64_t fg_launches = 0;

    // instrumentation: kernel launches issued, and CUDA-event timing of one kernel kind
    int64_t nlaunch = 0;
    int prof_kind = -1, prof_min_blocks = 0, prof_used = 0;
    int64_t prof_launches = 0, prof_cells = 0;
    std::vector<cudaEvent_t> prof_ev;
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int build_tables(ohm_hier *H, std::string &err) {
    const ohm_hier_desc &d = H->d;
    const int nlev = d.nlevels;
    H->amr.resize(nlev);
    // levels and block ranges
    int64_t pos = 0;
    for (int l = 0; l < nlev; l++) {
        HGrid &g = H->amr[l];
        g.level = l;
        for (int a = 0; a < 3; a++) {
            g.dims[a] = d.base_cells[a] << l;
            g.nb[a] = g.dims[a] / BS;
        }
        g.h = d.dx0 / (double)(1 << l);
        g.off = (int)pos;
        while (pos < H->nblocks && H->lijk[4 * pos] == l) {
            int bi = H->lijk[4 * pos + 1], bj = H->lijk[4 * pos + 2], bk = H->lijk[4 * pos + 3];
            if (bi < 0 || bj < 0 || bk < 0 || bi >= g.nb[0] || bj >= g.nb[1] || bk >= g.nb[2]) {
                err = "block " + std::to_string(pos) + " outside its level";
                return OHM_ERR_INVALID;
            }
            if (!g.index.emplace(key3(bi, bj, bk), g.n()).second) {
                err = "block " + std::to_string(pos) + " duplicated";
                return OHM_ERR_INVALID;
            }
            g.bijk.insert(g.bijk.end(), {bi, bj, bk});
            pos++;
        }
        if (g.n() == 0) {
            err = "level " + std::to_string(l) + " has no blocks";
            return OHM_ERR_INVALID;
        }
    }
    if (pos != H->nblocks) {
        err = "block list not sorted by level or level out of range";
        return OHM_ERR_INVALID;
    }
    if ((int64_t)H->amr[0].n() != (int64_t)H->amr[0].nb[0] * H->amr[0].nb[1] * H->amr[0].nb[2]) {
        err = "level 0 does not tile the base grid";
        return OHM_ERR_INVALID;
    }
    // octree completeness and proper nesting
    for (int l = 1; l < nlev; l++) {
        HGrid &g = H->amr[l], &p = H->amr[l - 1];
        for (int b = 0; b < g.n(); b++) {
            int bi = g.bijk[3 * b], bj = g.bijk[3 * b + 1], bk = g.bijk[3 * b + 2];
            int pi = bi >> 1, pj = bj >> 1, pk = bk >> 1;
            for (int o = 0; o < 8; o++)
                if (g.find(2 * pi + (o & 1), 2 * pj + ((o >> 1) & 1), 2 * pk + (o >> 2)) < 0) {
                    err = "level " + std::to_string(l) + ": incomplete octet";
                    return OHM_ERR_INVALID;
                }
            for (int dk = -1; dk <= 1; dk++)
                for (int dj = -1; dj <= 1; dj++)
                    for (int di = -1; di <= 1; di++)
                        if (p.find(pi + di, pj + dj, pk + dk) < 0) {
                            err = "level " + std::to_string(l) + ": not properly nested";
                            return OHM_ERR_INVALID;
                        }
        }
    }
    // per-level tables
    for (int l = 0; l < nlev; l++) {
        HGrid &g = H->amr[l];
        const int n = g.n();
        g.nbr.assign((size_t)n * 27, -1);
        g.covered.assign(n, 0);
        g.child.assign((size_t)n * 8, -1);
        g.parent.assign(n, -1);
        g.octant.assign(n, 0);
        g.origin = g.bijk;
        g.gslot.assign(n, -1);
        g.freg.assign((size_t)n * 6, -1);
        g.rsrc.assign((size_t)n * 6, -1);
        for (int b = 0; b < n; b++) {
            int bi = g.bijk[3 * b], bj = g.bijk[3 * b + 1], bk = g.bijk[3 * b + 2];
            for (int dk = -1; dk <= 1; dk++)
                for (int dj = -1; dj <= 1; dj++)
                    for (int di = -1; di <= 1; di++)
                        g.nbr[(size_t)b * 27 + (dk + 1) * 9 + (dj + 1) * 3 + di + 1] = g.find(bi + di, bj + dj, bk + dk);
            if (l + 1 < nlev) {
                const HGrid &f = H->amr[l + 1];
                for (int o = 0; o < 8; o++)
                    g.child[(size_t)b * 8 + o] = f.find(2 * bi + (o & 1), 2 * bj + ((o >> 1) & 1), 2 * bk + (o >> 2));
                g.covered[b] = g.child[(size_t)b * 8] >= 0;
            }
            if (l > 0) {
                g.parent[b] = H->amr[l - 1].find(bi >> 1, bj >> 1, bk >> 1);
                g.octant[b] = (uint8_t)((bi & 1) | ((bj & 1) << 1) | ((bk & 1) << 2));
                bool absent = false;
                for (int q = 0; q < 27; q++) {
                    int di = q % 3 - 1, dj = (q / 3) % 3 - 1, dk = q / 9 - 1;
                    if ((di != 0) + (dj != 0) + (dk != 0) == 3) continue;
                    if (g.nbr[(size_t)b * 27 + q] < 0) absent = true;
                }
                if (absent) {
                    g.gslot[b] = H->nslot++;
                    g.slot_block.push_back(b);
                }
                for (int s = 0; s < 6; s++) {
                    int a = s >> 1, hi = s & 1;
                    int dd[3] = {0, 0, 0};
                    dd[a] = hi ? 1 : -1;
                    if (g.nbr[(size_t)b * 27 + (dd[2] + 1) * 9 + (dd[1] + 1) * 3 + dd[0] + 1] < 0) g.freg[(size_t)b * 6 + s] = H->nreg++;
                }
            }
        }
        g.nslot = (int)g.slot_block.size();
        g.slot0 = H->nslot - g.nslot;
    }
    // reflux sources: leaf block faces next to a covered block take the four fine fluxes
    for (int l = 0; l + 1 < nlev; l++) {
        HGrid &g = H->amr[l];
        const HGrid &f = H->amr[l + 1];
        for (int b = 0; b < g.n(); b++) {
            if (g.covered[b]) continue;
            for (int s = 0; s < 6; s++) {
                int a = s >> 1, hi = s & 1;
                int dd[3] = {0, 0, 0};
                dd[a] = hi ? 1 : -1;
                int nb = g.nbr[(size_t)b * 27 + (dd[2] + 1) * 9 + (dd[1] + 1) * 3 + dd[0] + 1];
                if (nb < 0 || !g.covered[nb]) continue;
                int ax[2], q = 0;
                for (int c = 0; c < 3; c++)
                    if (c != a) ax[q++] = c;
                int ent = H->nrsrc++;
                g.rsrc[(size_t)b * 6 + s] = ent;
                for (int vb = 0; vb < 2; vb++)
                    for (int ub = 0; ub < 2; ub++) {
                        int o = 0;
                        o |= (hi ? 0 : 1) << a;
                        o |= ub << ax[0];
                        o |= vb << ax[1];
                        int ch = g.child[(size_t)nb * 8 + o];
                        int slot = ch >= 0 ? f.freg[(size_t)ch * 6 + 2 * a + (1 - hi)] : -1;
                        if (slot < 0) {
                            err = "internal: missing flux register at a coarse-fine face";
                            return OHM_ERR_INVALID;
                        }
                        H->rsrc_tab.push_back(slot);
                    }
            }
        }
    }
    // base multigrid grids: halve while every dimension is even and >= 4
    int dims[3] = {d.base_cells[0], d.base_cells[1], d.base_cells[2]};
    double h = d.dx0;
    bool blocked = true;
    while (dims[0] % 2 == 0 && dims[1] % 2 == 0 && dims[2] % 2 == 0 && dims[0] >= 4 && dims[1] >= 4 && dims[2] >= 4) {
        for (int a = 0; a < 3; a++) dims[a] /= 2;
        h *= 2.0;
        // mixed precision: a power-of-two grid of at most MIN_BLOCKED_CELLS cells and everything
        // below it go to the coarsest-grid solver, which holds them in shared memory
        const bool p2 = !(dims[0] & (dims[0] - 1)) && !(dims[1] & (dims[1] - 1)) && !(dims[2] & (dims[2] - 1));
        const bool to_bottom = H->mixed && p2 && (int64_t)dims[0] * dims[1] * dims[2] <= MIN_BLOCKED_CELLS;
        if (blocked && !to_bottom && dims[0] % BS == 0 && dims[1] % BS == 0 && dims[2] % BS == 0) {
            HGrid g;
            g.level = -1;
            g.h = h;
            for (int a = 0; a < 3; a++) {
                g.dims[a] = dims[a];
                g.nb[a] = dims[a] / BS;
            }
            std::vector<std::array<int, 3>> bl;
            for (int k = 0; k < g.nb[2]; k++)
                for (int j = 0; j < g.nb[1]; j++)
                    for (int i = 0; i < g.nb[0]; i++) bl.push_back({i, j, k});
            std::stable_sort(bl.begin(), bl.end(), [](const std::array<int, 3> &x, const std::array<int, 3> &y) {
                return morton(x[0], x[1], x[2]) < morton(y[0], y[1], y[2]);
            });
            for (auto &q : bl) {
                g.index.emplace(key3(q[0], q[1], q[2]), g.n());
                g.bijk.insert(g.bijk.end(), {q[0], q[1], q[2]});
            }
            const int n = g.n();
            g.nbr.assign((size_t)n * 27, -1);
            g.origin = g.bijk;
            g.parent.assign(n, -1);
            g.octant.assign(n, 0);
            for (int b = 0; b < n; b++) {
                int bi = g.bijk[3 * b], bj = g.bijk[3 * b + 1], bk = g.bijk[3 * b + 2];
                for (int q = 0; q < 27; q++)
                    g.nbr[(size_t)b * 27 + q] = g.find(bi + q % 3 - 1, bj + (q / 3) % 3 - 1, bk + q / 9 - 1);
            }
            H->mg.push_back(std::move(g));
        } else {
            blocked = false;
            if (H->small.size() >= (size_t)MAX_SMALL) {
                err = "too many coarse grids";
                return OHM_ERR_INVALID;
            }
            H->small.push_back({dims[0], dims[1], dims[2]});
        }
    }
    if (H->small.empty()) {
        err = "internal: no coarsest grid";
        return OHM_ERR_INVALID;
    }
    // parent / octant links from each blocked grid into the next blocked grid
    auto link = [](HGrid &fine, const HGrid &coarse) {
        for (int b = 0; b < fine.n(); b++) {
            int bi = fine.bijk[3 * b], bj = fine.bijk[3 * b + 1], bk = fine.bijk[3 * b + 2];
            fine.parent[b] = coarse.find(bi >> 1, bj >> 1, bk >> 1);
            fine.octant[b] = (uint8_t)((bi & 1) | ((bj & 1) << 1) | ((bk & 1) << 2));
        }
    };
    if (!H->mg.empty()) link(H->amr[0], H->mg[0]);
    for (size_t m = 0; m + 1 < H->mg.size(); m++) link(H->mg[m], H->mg[m + 1]);
    return OHM_OK;
}

// Batches: the tables of one instance (built above) repeated K times.  Every grid keeps its
// blocks instance after instance; block, slot, register and reflux-source indices of copy k
// are shifted by k times the per-instance count of the grid they point into.
void replicate(ohm_hier *H) {
    const int K = H->K;
    auto rep = [K](std::vector<int> &v, int per_block, int nb, int shift) {
        std::vector<int> o;
        o.reserve(v.size() * K);
        for (int k = 0; k < K; k++)
            for (size_t i = 0; i < (size_t)nb * per_block; i++) o.push_back(v[i] >= 0 ? v[i] + k * shift : -1);
        v.swap(o);
    };
    auto rep8 = [K](std::vector<uint8_t> &v) {
        std::vector<uint8_t> o;
        for (int k = 0; k < K; k++) o.insert(o.end(), v.begin(), v.end());
        v.swap(o);
    };
    const int nreg = H->nreg, nrsrc = H->nrsrc;
    std::vector<int> nb_amr, nb_mg, slot0_old, nslot_old;
    for (auto &g : H->amr) nb_amr.push_back(g.n());
    for (auto &g : H->mg) nb_mg.push_back(g.n());
    int slot_base = 0;
    for (size_t l = 0; l < H->amr.size(); l++) {
        HGrid &g = H->amr[l];
        const int nb = nb_amr[l];
        const int nb_child = l + 1 < H->amr.size() ? nb_amr[l + 1] : 0;
        const int nb_par = l > 0 ? nb_amr[l - 1] : (nb_mg.empty() ? 0 : nb_mg[0]);
        // ghost slots: copy k of local slot s is slot_base + k * nslot + s
        std::vector<int> gs;
        for (int k = 0; k < K; k++)
            for (int b = 0; b < nb; b++) gs.push_back(g.gslot[b] >= 0 ? slot_base + k * g.nslot + (g.gslot[b] - g.slot0) : -1);
        g.gslot.swap(gs);
        rep(g.slot_block, 1, g.nslot, nb);
        g.slot0 = slot_base;
        g.nslot *= K;
        slot_base += g.nslot;
        rep(g.nbr, 27, nb, nb);
        rep(g.child, 8, nb, nb_child);
        rep(g.parent, 1, nb, nb_par);
        rep(g.freg, 6, nb, nreg);
        rep(g.rsrc, 6, nb, nrsrc);
        rep(g.origin, 3, nb, 0);
        rep(g.bijk, 3, nb, 0);
        rep8(g.covered);
        rep8(g.octant);
        g.off *= K;
        g.inst_nblk = nb;
    }
    for (size_t m = 0; m < H->mg.size(); m++) {
        HGrid &g = H->mg[m];
        const int nb = nb_mg[m];
        const int nb_par = m + 1 < H->mg.size() ? nb_mg[m + 1] : 0;
        rep(g.nbr, 27, nb, nb);
        rep(g.parent, 1, nb, nb_par);
        rep(g.origin, 3, nb, 0);
        rep(g.bijk, 3, nb, 0);
        rep8(g.octant);
        g.inst_nblk = nb;
    }
    rep(H->rsrc_tab, 1, nrsrc * 4, nreg);
    H->nslot = slot_base;
    H->nreg = nreg * K;
    H->nrsrc = nrsrc * K;
    H->nblocks *= K;
    H->ranges.nlev = (int)H->amr.size();
    for (size_t l = 0; l < H->amr.size(); l++) {
        H->ranges.off[l] = H->amr[l].off;
        H->ranges.n[l] = nb_amr[l];
    }
}

template <typename V>
void push_table(std::vector<char> &blob, std::vector<size_t> &offs, const std::vector<V> &v) {
    size_t o = align256(blob.size());
    blob.resize(o + v.size() * sizeof(V));
    if (!v.empty()) memcpy(blob.data() + o, v.data(), v.size() * sizeof(V));
    offs.push_back(o);
}

int allocate(ohm_hier *H, std::string &err, int64_t *dry_bytes = nullptr) {
    const size_t tsz = H->mixed ? sizeof(float) : sizeof(double);
    const size_t n = (size_t)H->nblocks;
    // tables
    std::vector<char> blob;
    std::vector<size_t> offs;
    std::vector<HGrid *> grids;
    for (auto &g : H->amr) grids.push_back(&g);
    for (auto &g : H->mg) grids.push_back(&g);
    for (HGrid *g : grids) {
        push_table(blob, offs, g->nbr);
        push_table(blob, offs, g->covered);
        push_table(blob, offs, g->gslot);
        push_table(blob, offs, g->parent);
        push_table(blob, offs, g->octant);
        push_table(blob, offs, g->child);
        push_table(blob, offs, g->origin);
        push_table(blob, offs, g->freg);
        push_table(blob, offs, g->rsrc);
        push_table(blob, offs, g->slot_block);
    }
    push_table(blob, offs, H->rsrc_tab);
    // data
    size_t total = align256(blob.size());
    std::vector<std::pair<void **, size_t>> plan;
    auto want = [&](void **p, size_t bytes) { plan.push_back({p, bytes}); };
    want((void **)&H->S, n * 3 * B3 * 8);
    want((void **)&H->eta64, n * B3 * 8);
    want((void **)&H->Bscr, n * 3 * B3 * 8);
    want((void **)&H->ghostB, (size_t)H->nslot * 3 * T3 * 8);
    want((void **)&H->ghostEta64, (size_t)H->nslot * T3 * 8);
    want((void **)&H->reg, (size_t)H->nreg * 128 * 8);
    want((void **)&H->partials, n * 3 * 8);
    want((void **)&H->dnorm, 64);
    want((void **)&H->redscr, NORM_SCRATCH_BYTES);
    want(&H->ghostE, (size_t)H->nslot * 3 * T3 * tsz);
    if (H->mixed) want(&H->ghostEtaT, (size_t)H->nslot * T3 * tsz);
    want(&H->amrbuf.r, n * 3 * B3 * tsz);
    if (H->mixed) want(&H->rout, n * 3 * B3 * tsz);
    // the inner correction: float32 under mixed precision, float64 for the FP64 FGMRES
    if (H->mixed || H->d.krylov > 0) want(&H->eacc, n * 3 * B3 * tsz);
    {
        const int m = H->d.krylov;
        if (m > 0) {
            // Arnoldi basis and preconditioned vectors in the multigrid's precision
            for (int i = 0; i <= m; i++) want((void **)&H->kv[i], n * 3 * B3 * tsz);
            for (int i = 0; i < m; i++) want((void **)&H->kz[i], n * 3 * B3 * tsz);
            want((void **)&H->wblk, n * sizeof(double));
            const size_t K = (size_t)H->K;
            if (H->batched) {
                want((void **)&H->kpart, n * (KMAX + 1) * sizeof(double));
                want((void **)&H->kdots, K * (KMAX + 1) * sizeof(double));
                want((void **)&H->binst, n * sizeof(int));
            } else {
                want((void **)&H->kpart, ((n + 1) / 2) * (KMAX + 1) * sizeof(double));  // per block pair
                want((void **)&H->kdots, (KMAX + 1) * sizeof(double));
            }
            // batches: the FGMRES scalars of every instance on the device
            if (H->batched) want((void **)&H->kcoef, K * (KMAX + 1) * sizeof(float));
            if (H->batched) {
                want((void **)&H->fg.Hm, K * (KMAX + 1) * KMAX * sizeof(double));
                want((void **)&H->fg.cs, K * KMAX * sizeof(double));
                want((void **)&H->fg.sn, K * KMAX * sizeof(double));
                want((void **)&H->fg.g, K * (KMAX + 1) * sizeof(double));
                want((void **)&H->fg.beta0, K * 5 * sizeof(double));  // beta0, beta, brest, target, hn
                want((void **)&H->fg.cycles, K * 2 * sizeof(int) + sizeof(int));  // cycles, jend, any_need2
                want((void **)&H->fg.live, K * 6);  // live, arn, act, need2, run, compute mask
            }
        }
    }
    want(&H->amrbuf.e, n * 3 * B3 * tsz);
    want(&H->amrbuf.e2, n * 3 * B3 * tsz);
    want(&H->amrbuf.inv, n * 3 * B3 * tsz);
    if (H->mixed) want(&H->amrbuf.eta, n * B3 * tsz);
    H->mgbuf.resize(H->mg.size());
    for (size_t m = 0; m < H->mg.size(); m++) {
        size_t nb = (size_t)H->mg[m].n();
        want(&H->mgbuf[m].r, nb * 3 * B3 * tsz);
        want(&H->mgbuf[m].e, nb * 3 * B3 * tsz);
        want(&H->mgbuf[m].e2, nb * 3 * B3 * tsz);
        want(&H->mgbuf[m].inv, nb * 3 * B3 * tsz);
        want(&H->mgbuf[m].eta, nb * B3 * tsz);
    }
    if (H->batched) {
        want((void **)&H->eta_user, n * B3 * 8);
        want((void **)&H->bscale, n * 8);
        want((void **)&H->dnormK, (size_t)H->K * 4 * 8);
        want((void **)&H->imask_d, (size_t)H->K * 2);  // outer and inner masks
    }
    for (size_t q = 0; q < H->small.size(); q++) {
        size_t nc = (size_t)H->K * H->small[q][0] * H->small[q][1] * H->small[q][2];
        want(&H->smallbuf[q].r, nc * 3 * tsz);
        want(&H->smallbuf[q].e, nc * 3 * tsz);
        want(&H->smallbuf[q].e2, nc * 3 * tsz);
        want(&H->smallbuf[q].inv, nc * 3 * tsz);
        want(&H->smallbuf[q].eta, nc * tsz);
    }
    std::vector<size_t> doff;
    for (auto &p : plan) {
        doff.push_back(total);
        total += align256(p.second);
    }
    if (dry_bytes) {
        *dry_bytes = (int64_t)total;
        return OHM_OK;
    }
    if (cudaMalloc(&H->pool, total) != cudaSuccess) {
        cudaGetLastError();
        err = "device allocation of " + std::to_string(total) + " bytes failed";
        return OHM_ERR_OOM;
    }
    char *base = (char *)H->pool;
    for (size_t i = 0; i < plan.size(); i++) *plan[i].first = plan[i].second ? base + doff[i] : nullptr;
    H->d_err = (int *)(H->dnorm + 4);
    if (!H->mixed) {
        H->ghostEtaT = H->ghostEta64;
        H->amrbuf.eta = H->eta64;
    }
    if (cudaMemset(H->redscr, 0, NORM_SCRATCH_BYTES) != cudaSuccess ||
        cudaMemcpy(base, blob.data(), blob.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        err = "table upload failed";
        return OHM_ERR_CUDA;
    }
    if (cudaMallocHost((void **)&H->hnorm, 256) != cudaSuccess) {
        err = "pinned allocation failed";
        return OHM_ERR_OOM;
    }
    H->hdots = H->hnorm + 8;
    // the eta comparison's flag, the norms and the Krylov products, written by the kernels
    // straight into pinned host memory: the host then reads them after synchronising its stream,
    // without a copy that could wait behind another stream's large transfer
    if (cudaHostGetDevicePointer((void **)&H->hnorm_dev, H->hnorm, 0) != cudaSuccess) {
        cudaGetLastError();
        H->hnorm_dev = nullptr;
    }
    H->flag_dev = H->hnorm_dev ? reinterpret_cast<int *>(H->hnorm_dev + 24) : nullptr;
    if (H->batched) {
        if (cudaMallocHost((void **)&H->hnormK, (size_t)H->K * 4 * sizeof(double)) != cudaSuccess ||
            cudaMallocHost((void **)&H->imask_h, (size_t)H->K * 2) != cudaSuccess) {
            err = "pinned allocation failed";
            return OHM_ERR_OOM;
        }
        if (H->kcoef) {  // the instance of every block (the FGMRES state is set up below)
            std::vector<int> bi((size_t)H->nblocks, 0);
            for (int l = 0; l < H->ranges.nlev; l++)
                for (int q = 0; q < H->K; q++)
                    for (int b = 0; b < H->ranges.n[l]; b++) bi[(size_t)H->ranges.off[l] + (size_t)q * H->ranges.n[l] + b] = q;
            if (cudaMemcpy(H->binst, bi.data(), bi.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
                err = "table upload failed";
                return OHM_ERR_CUDA;
            }
        }
    }
    if (H->kcoef) {  // device FGMRES scalars (batches, mixed precision with krylov > 0)
        if (cudaMallocHost((void **)&H->fg_host, (size_t)H->K * 16) != cudaSuccess) {
            err = "pinned allocation failed";
            return OHM_ERR_OOM;
        }
        FgState &f = H->fg;
        const int K = H->K;
        f.beta = f.beta0 + K;
        f.brest = f.beta0 + 2 * K;
        f.target = f.beta0 + 3 * K;
        f.hn = f.beta0 + 4 * K;
        f.jend = f.cycles + K;
        f.any_need2 = f.cycles + 2 * K;
        f.arn = f.live + K;
        f.act = f.live + 2 * K;
        f.need2 = f.live + 3 * K;
        f.run = f.live + 4 * K;
        f.imask = f.live + 5 * K;  // compute mask of the V-cycle and operator launches
        f.dots = H->kdots;
        f.coef = H->kcoef;
        f.K = K;
        f.m = H->d.krylov;
        f.max_outer = H->d.max_outer;
    }
    if (H->wblk) {  // inner-product weights: h^3 on leaf blocks, 0 on covered ones
        std::vector<double> w((size_t)H->nblocks, 0.0);
        for (auto &g : H->amr)
            for (int b = 0; b < g.n(); b++) w[(size_t)g.off + b] = g.covered[b] ? 0.0 : g.h * g.h * g.h;
        if (cudaMemcpy(H->wblk, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            err = "weight upload failed";
            return OHM_ERR_CUDA;
        }
    }
    size_t k = 0;
    for (HGrid *g : grids) {
        GridDev &dv = g->dev;
        dv.nblk = g->n();
        dv.level_shift = g->level < 0 ? 0 : g->level;
        dv.h = g->h;
        for (int a = 0; a < 3; a++) dv.dims[a] = g->dims[a];
        auto ptr = [&](size_t o, bool nonempty) -> const void * { return nonempty ? base + o : nullptr; };
        dv.nbr = (const int *)ptr(offs[k + 0], !g->nbr.empty());
        dv.covered = (const uint8_t *)ptr(offs[k + 1], !g->covered.empty());
        dv.gslot = (const int *)ptr(offs[k + 2], !g->gslot.empty() && g->level > 0);
        dv.parent = (const int *)ptr(offs[k + 3], !g->parent.empty());
        dv.octant = (const uint8_t *)ptr(offs[k + 4], !g->octant.empty());
        dv.child = (const int *)ptr(offs[k + 5], !g->child.empty());
        dv.origin = (const int *)ptr(offs[k + 6], !g->origin.empty());
        dv.freg = (const int *)ptr(offs[k + 7], !g->freg.empty() && g->level > 0);
        bool anyr = std::any_of(g->rsrc.begin(), g->rsrc.end(), [](int v) { return v >= 0; });
        dv.rsrc = (const int *)ptr(offs[k + 8], anyr);
        dv.slot_block = (const int *)ptr(offs[k + 9], !g->slot_block.empty());
        dv.nslot = g->nslot;
        dv.slot0 = g->slot0;
        dv.inst_nblk = g->inst_nblk;
        const int nb = g->n();
        g->brick = nb % 2 == 0 && g->nslot == 0 && !g->nbr.empty() &&
                   std::none_of(g->nbr.begin(), g->nbr.end(), [](int v) { return v < 0; });
        for (int q = 0; g->brick && q < nb / 2; q++) g->brick = g->nbr[(size_t)(2 * q) * 27 + 14] == 2 * q + 1;
        k += 10;
    }
    H->d_rsrc = (int *)(H->rsrc_tab.empty() ? nullptr : base + offs[k]);
    // grids whose coarser multigrid grid holds their octets in order (Morton-ordered complete grids)
    auto set_octet = [](HGrid &f, const HGrid &c) {
        f.octet = f.n() == 8 * c.n() && c.nslot == 0 && !c.nbr.empty() &&
                  std::none_of(c.nbr.begin(), c.nbr.end(), [](int v) { return v < 0; });
        for (int b = 0; f.octet && b < f.n(); b++) f.octet = f.parent[b] == (b >> 3) && f.octant[b] == (b & 7);
    };
    if (!H->mg.empty()) set_octet(H->amr[0], H->mg[0]);
    for (size_t m = 0; m + 1 < H->mg.size(); m++) set_octet(H->mg[m], H->mg[m + 1]);
    return OHM_OK;
}

#define CK(x)                                 \
    do {                                      \
        cudaError_t e_ = (x);                 \
        if (e_ != cudaSuccess) return OHM_ERR_CUDA; \
    } while (0)

// Kernel launch with bookkeeping: counts the launch and, when this kernel kind is being
// timed and the launch covers at least prof_min_blocks blocks, brackets it with events.
inline int prof_begin(ohm_hier *H, int kind, int nblk) {
    if (H->prof_kind != kind || nblk < H->prof_min_blocks || H->prof_used + 2 > (int)H->prof_ev.size()) return -1;
    int i = H->prof_used;
    cudaEventRecord(H->prof_ev[i], H->s);
    return i;
}
inline void prof_end(ohm_hier *H, int i, int nblk) {
    H->nlaunch++;
    if (i < 0) return;
    cudaEventRecord(H->prof_ev[i + 1], H->s);
    H->prof_used += 2;
    H->prof_launches++;
    H->prof_cells += (int64_t)std::llround((double)nblk * B3 * (H->cmask ? H->active_frac : 1.0));
}
#define LAUNCH(H, kind, nblk, call)            \
    do {                                       \
        int pi_ = prof_begin((H), (kind), (nblk)); \
        cudaError_t e_ = (call);               \
        prof_end((H), pi_, (nblk));            \
        if (e_ != cudaSuccess) return OHM_ERR_CUDA; \
    } while (0)

template <typename T>
T *amr_ptr(void *p, const HGrid &g, int ncomp) {
    return (T *)p + (size_t)g.off * ncomp * B3;
}

template <typename T>
SmallDev<T> small_dev(ohm_hier *H) {
    SmallDev<T> sm;
    sm.n = (int)H->small.size();
    sm.ninst = H->K;
    sm.imask = H->cmask;
    sm.omega = H->d.omega;
    double h = H->d.dx0 * std::pow(2.0, (double)(H->mg.size() + 1));
    for (int q = 0; q < sm.n; q++) {
        for (int a = 0; a < 3; a++) sm.dims[q][a] = H->small[q][a];
        sm.h[q] = h;
        h *= 2.0;
        sm.e[q] = (T *)H->smallbuf[q].e;
        sm.r[q] = (T *)H->smallbuf[q].r;
        sm.t[q] = (T *)H->smallbuf[q].e2;
        sm.eta[q] = (T *)H->smallbuf[q].eta;
        sm.inv[q] = (T *)H->smallbuf[q].inv;
    }
    return sm;
}

// eta: level ghosts, the multigrid copies and the eta chain below level 0
template <typename T>
int eta_derive(ohm_hier *H) {
    cudaStream_t s = H->s;
    for (int l = 1; l < H->nlev; l++)
        CK((launch_ghost_fill<double, double>(H->amr[l].dev, H->amr[l - 1].dev, amr_ptr<double>(H->eta64, H->amr[l - 1], 1),
                                              1, H->ghostEta64, H->d_err, s)));
    if (H->mixed) {
        CK((launch_convert<double, T>(H->eta64, (T *)H->amrbuf.eta, (size_t)H->nblocks * B3, s)));
        CK((launch_convert<double, T>(H->ghostEta64, (T *)H->ghostEtaT, (size_t)H->nslot * T3, s)));
    }
    const HGrid *f = &H->amr[0];
    const T *fe = (const T *)H->amrbuf.eta;
    for (size_t m = 0; m < H->mg.size(); m++) {
        CK(launch_restrict<T>(f->dev, fe, 1, (T *)H->mgbuf[m].eta, nullptr, nullptr, s));
        f = &H->mg[m];
        fe = (const T *)H->mgbuf[m].eta;
    }
    CK(launch_restrict<T>(f->dev, fe, 1, nullptr, (T *)H->smallbuf[0].eta, H->small[0].data(), s));
    SmallDev<T> sm = small_dev<T>(H);
    CK(launch_small_setup<T>(sm, 0.0, true, s));
    H->inv_dt = NAN;
    return OHM_OK;
}

// inverse diagonals of the multigrid grids for lambda*dt.  The fused float32 sweeps and the
// shared-memory coarsest-grid solver form the diagonal from eta: with the fused smoother a float32
// hierarchy computes inverse diagonals only for the grids swept by colour passes (ghost slots) and
// for coarsest-grid paths that read them.
template <typename T>
int prepare_dt(ohm_hier *H, double dt) {
    const bool lean = std::is_same<T, float>::value && H->smoother == 0;
    if (H->inv_dt == dt && (H->inv_all || lean)) return OHM_OK;
    const double lamdt = H->d.lambda * dt;
    cudaStream_t s = H->s;
    // the relaxation factor is folded into the inverse diagonal (omega / (1 + alpha))
    for (auto &g : H->amr) {
        if (lean && g.nslot == 0) continue;
        GridDev d = g.dev;
        d.omega = H->d.omega;
        CK(launch_invdiag<T>(d, amr_ptr<T>(H->amrbuf.eta, g, 1), (const T *)H->ghostEtaT, lamdt,
                             amr_ptr<T>(H->amrbuf.inv, g, 3), s));
    }
    for (size_t m = 0; m < H->mg.size(); m++) {
        if (lean && H->mg[m].nslot == 0) continue;
        GridDev d = H->mg[m].dev;
        d.omega = H->d.omega;
        CK(launch_invdiag<T>(d, (const T *)H->mgbuf[m].eta, nullptr, lamdt, (T *)H->mgbuf[m].inv, s));
    }
    SmallDev<T> sm = small_dev<T>(H);
    bool small_lean = false;
    if constexpr (std::is_same<T, float>::value)
        small_lean = lean && (int64_t)sm.dims[0][0] * sm.dims[0][1] * sm.dims[0][2] <= MAX_BOTTOM_CELLS &&
                     bottom_in_shared(sm);
    if (!small_lean) CK(launch_small_setup<T>(sm, lamdt, false, s));
    H->inv_dt = dt;
    H->inv_all = !lean;
    return OHM_OK;
}

// the grid's device tables with the current compute mask (batched inner iterations)
GridDev gdev(const ohm_hier *H, const HGrid &g) {
    GridDev d = g.dev;
    d.imask = H->cmask;
    d.omega = H->d.omega;
    return d;
}

struct GridRef {
    const HGrid *g;
    void *e, *e2, *r, *eta, *inv;
    const void *Ge, *Geta;
};

template <typename T>
GridRef amr_ref(ohm_hier *H, int l, bool with_ghost) {
    const HGrid &g = H->amr[l];
    return GridRef{&g,
                   amr_ptr<T>(H->amrbuf.e, g, 3),
                   amr_ptr<T>(H->amrbuf.e2, g, 3),
                   amr_ptr<T>(H->amrbuf.r, g, 3),
                   amr_ptr<T>(H->amrbuf.eta, g, 1),
                   amr_ptr<T>(H->amrbuf.inv, g, 3),
                   with_ghost ? H->ghostE : nullptr,
                   H->ghostEtaT};
}

template <typename T>
GridRef base_ref(ohm_hier *H, int m) {  // m = 0: AMR level 0
    if (m == 0) return amr_ref<T>(H, 0, false);
    Buffers &b = H->mgbuf[m - 1];
    return GridRef{&H->mg[m - 1], b.e, b.e2, b.r, b.eta, b.inv, nullptr, nullptr};
}

template <typename T>
int sweeps(ohm_hier *H, const GridRef &G, int n, double lamdt, bool zero = false) {
    // zero: G.e holds no valid values yet and stands for e = 0 (the pre-smoothing of a level)
    const size_t bytes = (size_t)G.g->n() * 3 * B3 * sizeof(T);
    if (std::is_same<T, float>::value && G.g->nslot == 0 && H->smoother == 0) {
        // float32 grids with every neighbour: one fused red+black launch per sweep, on block
        // pairs where the grid's blocks pair up along x.  The buffers alternate so that the
        // last sweep writes G.e; a pair sweep from zero reads nothing for e, so neither a
        // memset nor a final copy is needed then.
        const bool zs = zero && G.g->brick;
        if (zero && (!zs || n == 0)) CK(cudaMemsetAsync(G.e, 0, bytes, H->s));
        for (int i = 0; i < n; i++) {
            const bool to_e = zs ? ((n - 1 - i) % 2 == 0) : (i & 1);
            const T *src = (const T *)(to_e ? G.e2 : G.e);
            T *dst = (T *)(to_e ? G.e : G.e2);
            if (G.g->brick)
                LAUNCH(H, OHM_K_SMOOTH, G.g->n(), launch_smooth_rb2(gdev(H, *G.g), i == 0 && zs ? nullptr : (const float *)src,
                                                                    (float *)dst, (const float *)G.r, (const float *)G.eta,
                                                                    lamdt, H->s));
            else
                LAUNCH(H, OHM_K_SMOOTH, G.g->n(), launch_smooth_rb<T>(gdev(H, *G.g), src, dst, (const T *)G.r, (const T *)G.eta, lamdt, H->s));
        }
        if (!zs && (n & 1)) CK(cudaMemcpyAsync(G.e, G.e2, bytes, cudaMemcpyDeviceToDevice, H->s));
        return OHM_OK;
    }
    if (zero) CK(cudaMemsetAsync(G.e, 0, bytes, H->s));
    for (int i = 0; i < n; i++) {
        LAUNCH(H, OHM_K_SMOOTH, G.g->n(), launch_smooth<T>(gdev(H, *G.g), (const T *)G.e, (T *)G.e2, (const T *)G.r, (const T *)G.eta, (const T *)G.inv,
                            (const T *)G.Ge, (const T *)G.Geta, lamdt, 0, H->s));
        LAUNCH(H, OHM_K_SMOOTH, G.g->n(), launch_smooth<T>(gdev(H, *G.g), (const T *)G.e2, (T *)G.e, (const T *)G.r, (const T *)G.eta, (const T *)G.inv,
                            (const T *)G.Ge, (const T *)G.Geta, lamdt, 1, H->s));
    }
    return OHM_OK;
}
// The V-cycle over the lexicographic grids below the last blocked one, for the restricted
// residual already in r of small grid 0.  Grids of more than MAX_BOTTOM_CELLS cells take
// grid-wide launches (the same arithmetic as the one-block solver); the one-block solver runs
// the remaining grids, or the coarsest grid gets its sweeps grid-wide when even that is large.
template <typename T>
int small_vcycle(ohm_hier *H, double lamdt, int npre, int npost, int ncoarse) {
    SmallDev<T> sm = small_dev<T>(H);
    int s0 = 0;
    while (s0 < sm.n && (int64_t)sm.dims[s0][0] * sm.dims[s0][1] * sm.dims[s0][2] > MAX_BOTTOM_CELLS) s0++;
    if (s0 == 0) {
        LAUNCH(H, OHM_K_BOTTOM, 0, launch_bottom<T>(sm, lamdt, npre, npost, ncoarse, H->s));
        return OHM_OK;
    }
    const size_t cells0 = (size_t)sm.dims[0][0] * sm.dims[0][1] * sm.dims[0][2];
    CK(cudaMemsetAsync(sm.e[0], 0, (size_t)sm.ninst * 3 * cells0 * sizeof(T), H->s));  // from e = 0
    const int top = std::min(s0, sm.n - 1);  // grids stepped grid-wide on the way down
    for (int g = 0; g < top; g++) {
        LAUNCH(H, OHM_K_BOTTOM, 0, launch_lex_sweeps<T>(sm, g, lamdt, npre, H->s));
        LAUNCH(H, OHM_K_BOTTOM, 0, launch_lex_resid_restrict<T>(sm, g, lamdt, H->s));
    }
    if (s0 < sm.n) {
        SmallDev<T> v = sm;  // grids s0 .. n-1
        v.n = sm.n - s0;
        for (int q = 0; q < v.n; q++) {
            for (int a = 0; a < 3; a++) v.dims[q][a] = sm.dims[s0 + q][a];
            v.h[q] = sm.h[s0 + q];
            v.e[q] = sm.e[s0 + q];
            v.r[q] = sm.r[s0 + q];
            v.t[q] = sm.t[s0 + q];
            v.eta[q] = sm.eta[s0 + q];
            v.inv[q] = sm.inv[s0 + q];
        }
        LAUNCH(H, OHM_K_BOTTOM, 0, launch_bottom<T>(v, lamdt, npre, npost, ncoarse, H->s));
    } else {
        LAUNCH(H, OHM_K_BOTTOM, 0, launch_lex_sweeps<T>(sm, sm.n - 1, lamdt, ncoarse, H->s));
    }
    for (int g = top - 1; g >= 0; g--) {
        LAUNCH(H, OHM_K_BOTTOM, 0, launch_lex_prolong<T>(sm, g, H->s));
        LAUNCH(H, OHM_K_BOTTOM, 0, launch_lex_sweeps<T>(sm, g, lamdt, npost, H->s));
    }
    return OHM_OK;
}

// Residual t = r - L e of a base-grid level and its restriction into the next blocked grid
// (coarse) or the first lexicographic grid (lex, dims ld); t_out receives t when not null.
// float32 brick grids whose children sit in Morton octets take the block-pair kernel.
template <typename T>
cudaError_t resid_restrict_base(ohm_hier *H, const HGrid &g, const T *e, const T *r, const T *eta, double lamdt,
                                T *t_out, T *coarse, T *lex, const int *ld) {
    if constexpr (std::is_same<T, float>::value) {
        if (g.brick && !lex && (!coarse || g.octet))
            return launch_pair_op(gdev(H, g), e, r, eta, -lamdt / (2.0 * g.h * g.h), false, t_out, coarse, H->s);
    }
    return launch_resid_restrict<T>(gdev(H, g), e, r, eta, nullptr, nullptr, lamdt, t_out, coarse, lex, ld, H->s);
}

template <typename T>
int base_vcycle(ohm_hier *H, int m, double lamdt) {
    const ohm_hier_desc &d = H->d;
    GridRef G = base_ref<T>(H, m);
    int st;
    // level 0 takes nu_pre / nu_post, its coarsenings the coarse-grid counts when those are set
    const bool cs = m >= 1 && (d.nu_coarse_pre || d.nu_coarse_post);
    const int npre = cs ? d.nu_coarse_pre : d.nu_pre, npost = cs ? d.nu_coarse_post : d.nu_post;
    if ((st = sweeps<T>(H, G, npre, lamdt, true))) return st;  // the level's correction starts at 0
    const bool next_blocked = m < (int)H->mg.size();
    if (next_blocked) {
        GridRef C = base_ref<T>(H, m + 1);
        LAUNCH(H, OHM_K_RESID_RESTRICT, G.g->n(),
               resid_restrict_base<T>(H, *G.g, (const T *)G.e, (const T *)G.r, (const T *)G.eta, lamdt, nullptr, (T *)C.r,
                                      nullptr, nullptr));
        if ((st = base_vcycle<T>(H, m + 1, lamdt))) return st;
        if (G.g->octet)
            LAUNCH(H, OHM_K_PROLONG, G.g->n(), launch_prolong_add8<T>(gdev(H, *C.g), (const T *)C.e, (T *)G.e, H->s));
        else
            LAUNCH(H, OHM_K_PROLONG, G.g->n(), launch_prolong_add<T>(gdev(H, *G.g), &C.g->dev, (const T *)C.e, nullptr, nullptr, (T *)G.e, H->d_err, H->s));
    } else {
        LAUNCH(H, OHM_K_RESID_RESTRICT, G.g->n(), launch_resid_restrict<T>(gdev(H, *G.g), (const T *)G.e, (const T *)G.r, (const T *)G.eta, nullptr, nullptr, lamdt,
                                    nullptr, nullptr, (T *)H->smallbuf[0].r, H->small[0].data(), H->s));
        const bool csb = d.nu_coarse_pre || d.nu_coarse_post;  // the small grids are all coarser than level 0
        if ((st = small_vcycle<T>(H, lamdt, csb ? d.nu_coarse_pre : d.nu_pre, csb ? d.nu_coarse_post : d.nu_post,
                                  d.n_coarse)))
            return st;
        LAUNCH(H, OHM_K_PROLONG, G.g->n(), launch_prolong_add<T>(gdev(H, *G.g), nullptr, nullptr, (const T *)H->smallbuf[0].e, H->small[0].data(), (T *)G.e,
                                 H->d_err, H->s));
    }
    return sweeps<T>(H, G, npost, lamdt);
}

// One correction-scheme V-cycle over the AMR levels and the base grid.  r on leaf blocks
// holds the composite residual; the correction is left in e (all levels).
template <typename T>
int vcycle(ohm_hier *H, double lamdt) {
    const ohm_hier_desc &d = H->d;
    int st;
    for (int l = H->nlev - 1; l >= 1; l--) {
        GridRef G = amr_ref<T>(H, l, true);
        const HGrid &g = *G.g;
        if (g.nslot) CK(cudaMemsetAsync((T *)H->ghostE + (size_t)g.slot0 * 3 * T3, 0, (size_t)g.nslot * 3 * T3 * sizeof(T), H->s));
        if ((st = sweeps<T>(H, G, d.nu_pre, lamdt, true))) return st;  // from e = 0
        GridRef C = amr_ref<T>(H, l - 1, true);
        LAUNCH(H, OHM_K_RESID_RESTRICT, g.n(), launch_resid_restrict<T>(gdev(H, g), (const T *)G.e, (const T *)G.r, (const T *)G.eta, (const T *)G.Ge,
                                    (const T *)G.Geta, lamdt, nullptr, (T *)C.r, nullptr, nullptr, H->s));
    }
    if ((st = base_vcycle<T>(H, 0, lamdt))) return st;  // level 0 starts from e = 0 inside
    for (int l = 1; l < H->nlev; l++) {
        GridRef G = amr_ref<T>(H, l, true);
        GridRef C = amr_ref<T>(H, l - 1, true);
        LAUNCH(H, OHM_K_PROLONG, G.g->n(), launch_prolong_add<T>(gdev(H, *G.g), &C.g->dev, (const T *)C.e, nullptr, nullptr, (T *)G.e, H->d_err, H->s));
        LAUNCH(H, OHM_K_GHOST, G.g->nslot, (launch_ghost_fill<T, T>(gdev(H, *G.g), C.g->dev, (const T *)C.e, 3, (T *)H->ghostE, H->d_err, H->s)));
        if ((st = sweeps<T>(H, G, d.nu_post, lamdt))) return st;
    }
    return OHM_OK;
}

int sync_down(ohm_hier *H, double *B) {
    for (int l = H->nlev - 2; l >= 0; l--)
        LAUNCH(H, OHM_K_SYNC_DOWN, H->amr[l].n(), launch_sync_down(gdev(H, H->amr[l]), amr_ptr<double>(B, H->amr[l], 3), amr_ptr<double>(B, H->amr[l + 1], 3), H->s));
    return OHM_OK;
}

int fill_ghosts_B(ohm_hier *H, const double *B) {
    for (int l = 1; l < H->nlev; l++)
        LAUNCH(H, OHM_K_GHOST, H->amr[l].nslot, (launch_ghost_fill<double, double>(gdev(H, H->amr[l]), H->amr[l - 1].dev,
                                              amr_ptr<double>((void *)B, H->amr[l - 1], 3), 3, H->ghostB, H->d_err, H->s)));
    return OHM_OK;
}

// out = a X + c divF(X) + d Y on leaf blocks of every level (finest first, so refluxed
// fine fluxes are in the registers before the coarser level reads them), computed in TC.
template <typename TC, typename TO>
int composite_t(ohm_hier *H, const TC *X, const TC *Y, const TC *eta, const TC *Gx, const TC *Geta, double a, double c,
                double dcoef, TO *out, TO *out2, bool norms, double *outS = nullptr, double c2 = 0.0, bool ff64 = false) {
    for (int l = H->nlev - 1; l >= 0; l--) {
        const HGrid &g = H->amr[l];
        double vol = g.h * g.h * g.h;
        const size_t o3 = (size_t)g.off * 3 * B3;
        if constexpr (std::is_same<TC, double>::value && std::is_same<TO, float>::value) {
          if (ff64) {
            // an intermediate outer residual of OHM_MIXED: float-float arithmetic, Y in float64
            LAUNCH(H, OHM_K_COMPOSITE, g.n(),
                   launch_composite_df(gdev(H, g), X + o3, Y ? Y + o3 : nullptr, eta + (size_t)g.off * B3, Gx, Geta, a,
                                       c, dcoef, out + o3, out2 ? out2 + o3 : nullptr, H->reg, H->d_rsrc,
                                       norms ? H->partials + (size_t)g.off * 3 : nullptr, vol, H->s));
            continue;
          }
          if (H->ff) {
            // outer residual of OHM_MIXED_FF: float-float arithmetic, Y and outS hold the source
            // in float-float form
            LAUNCH(H, OHM_K_COMPOSITE, g.n(),
                   (launch_composite_df(gdev(H, g), X + o3, Y ? reinterpret_cast<const dfloat *>(Y) + o3 : nullptr,
                                        eta + (size_t)g.off * B3, Gx, Geta, a, c, dcoef, out + o3,
                                        out2 ? out2 + o3 : nullptr, H->reg, H->d_rsrc,
                                        norms ? H->partials + (size_t)g.off * 3 : nullptr, vol, H->s,
                                        outS ? reinterpret_cast<dfloat *>(outS) + o3 : nullptr, c2)));
            continue;
          }
        }
        if constexpr (std::is_same<TC, float>::value && std::is_same<TO, float>::value) {
            // the float32 operator (a = 1, d = 0, no Y) or residual (a = -1, d = 1) of a single-level
            // brick grid without norms: block-pair kernel
            const bool apply = !Y && a == 1.0 && dcoef == 0.0, resid = Y && a == -1.0 && dcoef == 1.0;
            if (H->nlev == 1 && g.brick && !norms && !out2 && !outS && (apply || resid)) {
                LAUNCH(H, OHM_K_COMPOSITE, g.n(),
                       launch_pair_op(gdev(H, g), X + o3, Y ? Y + o3 : nullptr, eta + (size_t)g.off * B3,
                                      c / (2.0 * g.h * g.h), apply, out + o3, nullptr, H->s));
                continue;
            }
        }
        {
            LAUNCH(H, OHM_K_COMPOSITE, g.n(),
                   (launch_composite<TC, TO>(gdev(H, g), X + o3, Y ? Y + o3 : nullptr, eta + (size_t)g.off * B3, Gx, Geta,
                                             a, c, dcoef, out + o3, out2 ? out2 + o3 : nullptr, H->reg, H->d_rsrc,
                                             norms ? H->partials + (size_t)g.off * 3 : nullptr, vol, H->s,
                                             outS ? outS + o3 : nullptr, c2)));
        }
    }
    if (norms) {
        if (H->batched)
            LAUNCH(H, OHM_K_NORM, 0, launch_norm_inst(H->partials, H->ranges, H->K, H->dnormK, H->s));
        else
            LAUNCH(H, OHM_K_NORM, 0, launch_norm_reduce(H->partials, (int)H->nblocks, H->redscr, H->dnorm, H->s,
                                                        H->hnorm_dev, H->d_err));
    }
    return OHM_OK;
}

// float64 composite operator on B-like fields (eta and ghosts of the state)
template <typename TO>
int composite(ohm_hier *H, const double *X, const double *Y, double a, double c, double dcoef, TO *out, bool norms,
              TO *out2 = nullptr, bool ff64 = false) {
    return composite_t<double, TO>(H, X, Y, H->eta64, H->ghostB, H->ghostEta64, a, c, dcoef, out, out2, norms, nullptr,
                                   0.0, ff64);
}

// The first residual of a step and its source from one flux divergence of b (Eqs. 14, 20):
// S = b - (1 - lambda) dt divF(b) into H->S, and R = S - L b = -dt divF(b) into out (and out2),
// with the norms of R against S.
template <typename TO>
int source_and_residual(ohm_hier *H, const double *b, double lam, double dt, TO *out, TO *out2) {
    return composite_t<double, TO>(H, b, nullptr, H->eta64, H->ghostB, H->ghostEta64, 1.0, -(1.0 - lam) * dt, 0.0, out,
                                   out2, true, H->S, -dt);
}

template <typename T>
int sync_down_t(ohm_hier *H, T *x) {
    for (int l = H->nlev - 2; l >= 0; l--)
        LAUNCH(H, OHM_K_SYNC_DOWN, H->amr[l].n(),
               launch_sync_down<T>(gdev(H, H->amr[l]), amr_ptr<T>(x, H->amr[l], 3), amr_ptr<T>(x, H->amr[l + 1], 3), H->s));
    return OHM_OK;
}

template <typename T>
int fill_ghosts_t(ohm_hier *H, const T *x, T *ghost) {
    for (int l = 1; l < H->nlev; l++)
        LAUNCH(H, OHM_K_GHOST, H->amr[l].nslot,
               (launch_ghost_fill<T, T>(gdev(H, H->amr[l]), H->amr[l - 1].dev, amr_ptr<T>((void *)x, H->amr[l - 1], 3), 3,
                                        ghost, H->d_err, H->s)));
    return OHM_OK;
}

// The error word alone, for operations that end without a norm reduction.
int read_err(ohm_hier *H, int *err_flag) {
    CK(cudaMemcpyAsync(H->hnorm + 4, H->d_err, sizeof(int), cudaMemcpyDeviceToHost, H->s));
    CK(cudaStreamSynchronize(H->s));
    memcpy(err_flag, &H->hnorm[4], sizeof(int));
    return OHM_OK;
}

// The norms of the last norm reduction and the error word as that reduction saw it (the
// reduction must be the last kernel on the stream that can set the error word).
int read_norms(ohm_hier *H, double out[4], int *err_flag) {
    // the norm kernel wrote its sums and the error word into hnorm when it is mapped
    if (!H->hnorm_dev) CK(cudaMemcpyAsync(H->hnorm, H->dnorm, 40, cudaMemcpyDeviceToHost, H->s));
    CK(cudaStreamSynchronize(H->s));
    double sr = H->hnorm[0], ss = H->hnorm[1];
    out[0] = ss > 0 ? std::sqrt(sr / ss) : std::sqrt(sr);
    out[1] = H->hnorm[2];
    out[2] = std::sqrt(sr);
    out[3] = std::sqrt(ss);
    int e;
    memcpy(&e, &H->hnorm[4], sizeof(int));
    *err_flag = e;
    return OHM_OK;
}

template <typename T>
int update_all(ohm_hier *H, double *B, const T *e, const uint8_t *imask = nullptr) {
    for (auto &g : H->amr)
        LAUNCH(H, OHM_K_UPDATE, g.n(), launch_update<T>(g.dev, amr_ptr<double>(B, g, 3), amr_ptr<T>((void *)e, g, 3), imask, H->s));
    return OHM_OK;
}

template <typename T>
int inner_fgmres(ohm_hier *H, double lamdt, double target, int *cycles);

template <typename T>
int cn_step_impl(ohm_hier *H, double *B, double dt, double tol, ohm_step_stats *stats) {
    const double lam = H->d.lambda, lamdt = lam * dt;
    int st;
    if ((st = prepare_dt<T>(H, dt))) return st;
    CK(cudaMemsetAsync(H->d_err, 0, sizeof(int), H->s));
    if ((st = sync_down(H, B))) return st;
    if ((st = fill_ghosts_B(H, B))) return st;
    H->has_S = true;
    H->last_dt = dt;
    int it = 0;
    double nr[4] = {0, 0, 0, 0}, first = 0;
    int result = OHM_OK;
    for (;;) {
        // the first residual comes with the source S from one flux divergence of b
        if ((st = it == 0 ? source_and_residual<T>(H, B, lam, dt, (T *)H->amrbuf.r, (T *)nullptr)
                          : composite<T>(H, B, H->S, -1.0, -lamdt, 1.0, (T *)H->amrbuf.r, true)))
            return st;
        int ef = 0;
        if ((st = read_norms(H, nr, &ef))) return st;
        if (ef) return OHM_ERR_INVALID;
        if (it == 0) first = nr[0];
        if (!std::isfinite(nr[0]) || !std::isfinite(nr[1])) {
            result = OHM_ERR_NONFINITE;
            break;
        }
        if (tol >= 0 && nr[0] <= tol) break;
        if (it >= H->d.max_outer) {
            result = tol >= 0 ? OHM_ERR_NOT_CONVERGED : OHM_OK;
            break;
        }
        if (H->d.krylov > 0) {
            // FGMRES in float64, right-preconditioned by the V-cycle, to the tolerance in one
            // solve (no float32 limit to stop at); `it` counts its V-cycles
            const double target = tol >= 0 ? 0.3 * tol / std::max(nr[0], 1e-300) : 0.0;
            if ((st = inner_fgmres<T>(H, lamdt, target, &it))) return st;
            if ((st = update_all<T>(H, B, (const T *)H->eacc))) return st;
        } else {
            if ((st = vcycle<T>(H, lamdt))) return st;
            if ((st = update_all<T>(H, B, (const T *)H->amrbuf.e))) return st;
            it++;
        }
        if ((st = sync_down(H, B))) return st;
        if ((st = fill_ghosts_B(H, B))) return st;
    }
    if (stats) {
        stats->cycles = it;
        stats->converged = (result == OHM_OK && tol >= 0) ? 1 : 0;
        stats->rel_l2_initial = first;
        stats->rel_l2 = nr[0];
        stats->max_abs = nr[1];
    }
    return result;
}

// Mixed precision as iterative refinement around Eqs. 16-18: the float64 residual
// R = S - L B is handed to a float32 multigrid solve of L e = R (V-cycles, each followed by
// the float32 composite residual of the correction equation) until that inner residual has
// dropped by max(inner_tol, 0.3 tol / ||R||/||S||) (inner_tol 1e-5 unless the descriptor sets
// it), then B += e in float64.  max_outer bounds the total number of V-cycles of the step.
constexpr double INNER_FLOOR_DEFAULT = 1e-5;

double inner_floor(const ohm_hier *H) { return H->d.inner_tol > 0 ? H->d.inner_tol : INNER_FLOOR_DEFAULT; }


// Weighted inner products <w, v_i> (i < S.k) and <w, w>, read back to the host.
int mdot(ohm_hier *H, const float *w, const VecSet &S, double *out) {
    LAUNCH(H, OHM_K_KRYLOV, (int)H->nblocks, launch_mdot(w, S, H->wblk, (int)H->nblocks, H->kpart, H->kdots, H->s, nullptr,
                                                         H->hnorm_dev ? H->hnorm_dev + 8 : nullptr));
    if (!H->hnorm_dev)
        CK(cudaMemcpyAsync(H->hdots, H->kdots, (S.k + 1) * sizeof(double), cudaMemcpyDeviceToHost, H->s));
    CK(cudaStreamSynchronize(H->s));
    memcpy(out, H->hdots, (S.k + 1) * sizeof(double));
    return OHM_OK;
}

// L x for a float32 field (covered cells first set from their children, ghosts filled)
int apply_L32(ohm_hier *H, float *x, const float *y, double a, double c, double d, float *out, double lamdt) {
    (void)lamdt;
    int st;
    if ((st = sync_down_t<float>(H, x))) return st;
    if ((st = fill_ghosts_t<float>(H, x, (float *)H->ghostE))) return st;
    return composite_t<float, float>(H, x, y, (const float *)H->amrbuf.eta, (const float *)H->ghostE,
                                     (const float *)H->ghostEtaT, a, c, d, out, (float *)nullptr, false);
}

// float64 counterparts of the Krylov helpers (the FP64 FGMRES)
template <typename T>
struct VecSetSel {
    using type = VecSet;
};
template <>
struct VecSetSel<double> {
    using type = VecSetD;
};
template <typename T>
using VecSetOf = typename VecSetSel<T>::type;

int mdot(ohm_hier *H, const double *w, const VecSetD &S, double *out) {
    LAUNCH(H, OHM_K_KRYLOV, (int)H->nblocks, launch_mdot(w, S, H->wblk, (int)H->nblocks, H->kpart, H->kdots, H->s,
                                                         H->hnorm_dev ? H->hnorm_dev + 8 : nullptr));
    if (!H->hnorm_dev)
        CK(cudaMemcpyAsync(H->hdots, H->kdots, (S.k + 1) * sizeof(double), cudaMemcpyDeviceToHost, H->s));
    CK(cudaStreamSynchronize(H->s));
    memcpy(out, H->hdots, (S.k + 1) * sizeof(double));
    return OHM_OK;
}

// out = a x + c divF(x) + d y for a float64 correction field (ghosts of x, the state's eta)
int apply_L64(ohm_hier *H, double *x, const double *y, double a, double c, double d, double *out) {
    int st;
    if ((st = sync_down_t<double>(H, x))) return st;
    if ((st = fill_ghosts_t<double>(H, x, (double *)H->ghostE))) return st;
    return composite_t<double, double>(H, x, y, H->eta64, (const double *)H->ghostE, H->ghostEta64, a, c, d, out,
                                       (double *)nullptr, false);
}

int apply_Lt(ohm_hier *H, float *x, const float *y, double a, double c, double d, float *out, double lamdt) {
    return apply_L32(H, x, y, a, c, d, out, lamdt);
}
int apply_Lt(ohm_hier *H, double *x, const double *y, double a, double c, double d, double *out, double) {
    return apply_L64(H, x, y, a, c, d, out);
}

int apply_mdot(ohm_hier *H, const double *z, double *w, const VecSetD &S, double lamdt, double *out) {
    int st;
    if ((st = apply_L64(H, const_cast<double *>(z), nullptr, 1.0, lamdt, 0.0, w))) return st;
    return mdot(H, w, S, out);
}

// w = L z with its products <w, v_i> (i < S.k) and <w, w>: in one pass on block pairs where the
// hierarchy is one brick grid, else the operator followed by the multi-dot.
int apply_mdot(ohm_hier *H, const float *z, float *w, const VecSet &S, double lamdt, double *out) {
    const HGrid &g = H->amr[0];
    if (H->nlev == 1 && g.brick && !H->batched) {
        LAUNCH(H, OHM_K_COMPOSITE, g.n(),
               launch_pair_apply_dots(gdev(H, g), z, (const float *)H->amrbuf.eta, lamdt / (2.0 * g.h * g.h), w, S,
                                      g.h * g.h * g.h, H->kpart, H->kdots, H->hnorm_dev ? H->hnorm_dev + 8 : nullptr,
                                      H->s));
        if (!H->hnorm_dev)
            CK(cudaMemcpyAsync(H->hdots, H->kdots, (S.k + 1) * sizeof(double), cudaMemcpyDeviceToHost, H->s));
        CK(cudaStreamSynchronize(H->s));
        memcpy(out, H->hdots, (S.k + 1) * sizeof(double));
        return OHM_OK;
    }
    int st;
    if ((st = apply_L32(H, const_cast<float *>(z), nullptr, 1.0, lamdt, 0.0, w, lamdt))) return st;
    return mdot(H, w, S, out);
}

// Inner solve of L x = R by FGMRES(m) (Saad 1993), right-preconditioned by one V-cycle per
// Arnoldi step, classical Gram-Schmidt in the leaf-volume inner product, Givens rotations on
// the host, restarts from the true residual: in float32 for mixed precision (R = rout, the
// float32 copy of the outer residual), in float64 for OHM_FP64 (R = the float64 residual).
// Stops when the residual has dropped by `target`, when a whole restart cycle gained less than
// a factor 2 (float32 has nothing more to give), or when the step's V-cycle budget is used.  x
// is left in eacc.
template <typename T>
int inner_fgmres(ohm_hier *H, double lamdt, double target, int *cycles) {
    const int m = H->d.krylov;
    const size_t nel = (size_t)H->nblocks * 3 * B3;
    // right-hand side: the float32 copy of the outer residual, or the float64 residual itself
    T *x = (T *)H->eacc, *rhs = (T *)(std::is_same<T, float>::value ? H->rout : H->amrbuf.r);
    int st;
    // x starts at 0: the first solution update writes Z y without reading x, and x is cleared
    // only if the solve ends before any update
    bool x_set = false;
    double nn[KMAX + 1];
    VecSetOf<T> none;
    none.k = 0;
    if ((st = mdot(H, rhs, none, nn))) return st;
    const double beta0 = std::sqrt(nn[0]);
    if (!(beta0 > 0) || !std::isfinite(beta0)) {
        CK(cudaMemsetAsync(x, 0, nel * sizeof(T), H->s));
        return OHM_OK;
    }
    double beta = beta0, beta_restart = beta0;
    LAUNCH(H, OHM_K_KRYLOV, (int)H->nblocks, launch_maxpy((T *)H->kv[0], rhs, none, (T)(1.0 / beta), nel, H->s));
    std::vector<double> Hm((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    auto h = [&](int i, int j) -> double & { return Hm[(size_t)i * m + j]; };
    for (;;) {
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int jend = 0;
        bool done = false;
        for (int j = 0; j < m && *cycles < H->d.max_outer; j++) {
            // z_j = V-cycle applied to v_j (the cycle's right-hand side and correction buffers
            // are pointed at v_j and z_j)
            void *r_save = H->amrbuf.r, *e_save = H->amrbuf.e;
            H->amrbuf.r = H->kv[j];
            H->amrbuf.e = H->kz[j];
            st = vcycle<T>(H, lamdt);
            H->amrbuf.r = r_save;
            H->amrbuf.e = e_save;
            if (st) return st;
            (*cycles)++;
            // w = L z_j, orthogonalised against v_0..v_j
            VecSetOf<T> S;
            S.k = j + 1;
            for (int i = 0; i <= j; i++) S.v[i] = (const T *)H->kv[i];
            if ((st = apply_mdot(H, (const T *)H->kz[j], (T *)H->kv[j + 1], S, lamdt, nn))) return st;
            double proj = 0.0;
            for (int i = 0; i <= j; i++) {
                h(i, j) = nn[i];
                S.c[i] = (T)nn[i];
                proj += nn[i] * nn[i];
            }
            // ||w - sum h_i v_i||^2 = <w,w> - sum h_i^2 for orthonormal v_i: when that keeps more
            // than 1% of <w,w> the orthogonalisation and the normalisation are one pass,
            // otherwise the norm is measured after orthogonalising.  The pass that forms
            // v_{j+1} (or scales it) is issued only when another Arnoldi step follows: after
            // the last step of a restart cycle, or one that met the target, v_{j+1} is never read.
            const double ww = nn[j + 1];
            double hn;
            const bool one_pass = ww - proj > 0.01 * ww;
            if (one_pass) {
                hn = std::sqrt(ww - proj);
            } else {
                LAUNCH(H, OHM_K_KRYLOV, (int)H->nblocks, launch_maxpy((T *)H->kv[j + 1], (T *)H->kv[j + 1], S, T(1), nel, H->s));
                if ((st = mdot(H, (const T *)H->kv[j + 1], none, nn))) return st;
                hn = std::sqrt(std::max(nn[0], 0.0));
            }
            h(j + 1, j) = hn;
            // Givens rotations
            for (int i = 0; i < j; i++) {
                double t = cs[i] * h(i, j) + sn[i] * h(i + 1, j);
                h(i + 1, j) = -sn[i] * h(i, j) + cs[i] * h(i + 1, j);
                h(i, j) = t;
            }
            double den = std::hypot(h(j, j), h(j + 1, j));
            cs[j] = den > 0 ? h(j, j) / den : 1.0;
            sn[j] = den > 0 ? h(j + 1, j) / den : 0.0;
            h(j, j) = den;
            h(j + 1, j) = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            jend = j + 1;
            if (std::fabs(g[j + 1]) <= target * beta0 || !(hn > 0)) {
                done = true;
                break;
            }
            if (j + 1 < m && *cycles < H->d.max_outer) {  // v_{j+1} for the next Arnoldi step
                if (one_pass)
                    LAUNCH(H, OHM_K_KRYLOV, (int)H->nblocks, launch_maxpy((T *)H->kv[j + 1], (T *)H->kv[j + 1], S, (T)(1.0 / hn), nel, H->s));
                else
                    LAUNCH(H, OHM_K_KRYLOV, (int)H->nblocks, launch_maxpy((T *)H->kv[j + 1], (T *)H->kv[j + 1], none, (T)(1.0 / hn), nel, H->s));
            }
        }
        // x += sum y_i z_i with R y = g
        for (int i = jend - 1; i >= 0; i--) {
            double s = g[i];
            for (int k = i + 1; k < jend; k++) s -= h(i, k) * y[k];
            y[i] = h(i, i) != 0 ? s / h(i, i) : 0.0;
        }
        if (jend > 0) {
            VecSetOf<T> Z;
            Z.k = jend;
            for (int i = 0; i < jend; i++) {
                Z.v[i] = (const T *)H->kz[i];
                Z.c[i] = (T)(-y[i]);
            }
            LAUNCH(H, OHM_K_KRYLOV, (int)H->nblocks, launch_maxpy(x, x_set ? x : nullptr, Z, T(1), nel, H->s));
            x_set = true;
        }
        if (done || *cycles >= H->d.max_outer || jend == 0) break;
        // restart from the true residual rhs - L x
        if ((st = apply_Lt(H, x, rhs, -1.0, -lamdt, 1.0, (T *)H->kv[0], lamdt))) return st;
        if ((st = mdot(H, (const T *)H->kv[0], none, nn))) return st;
        beta = std::sqrt(std::max(nn[0], 0.0));
        if (beta <= target * beta0 || !(beta > 0) || beta > 0.5 * beta_restart) break;
        beta_restart = beta;
        LAUNCH(H, OHM_K_KRYLOV, (int)H->nblocks, launch_maxpy((T *)H->kv[0], (T *)H->kv[0], none, (T)(1.0 / beta), nel, H->s));
    }
    if (!x_set) CK(cudaMemsetAsync(x, 0, nel * sizeof(T), H->s));
    return OHM_OK;
}

int cn_step_mixed(ohm_hier *H, double *B, double dt, double tol, ohm_step_stats *stats) {
    using T = float;
    const double lam = H->d.lambda, lamdt = lam * dt;
    int st;
    if ((st = prepare_dt<T>(H, dt))) return st;
    CK(cudaMemsetAsync(H->d_err, 0, sizeof(int), H->s));
    if ((st = sync_down(H, B))) return st;
    if ((st = fill_ghosts_B(H, B))) return st;
    H->has_S = true;
    H->last_dt = dt;
    T *r = (T *)H->amrbuf.r, *e = (T *)H->amrbuf.e, *rout = (T *)H->rout, *eacc = (T *)H->eacc;
    const size_t nbytes = (size_t)H->nblocks * 3 * B3 * sizeof(T);
    int cycles = 0, result = OHM_OK;
    double nr[4] = {0, 0, 0, 0}, first = 0;
    // OHM_MIXED_FF_CHECKED: the source and the first residual are float64, and so is every
    // residual that ends the step; an outer residual that the last correction is not expected to
    // bring below tol only sets the next inner solve's right-hand side, and is evaluated in
    // float-float (error about 2^-48 of the operands, far below any tol it is compared with).  A
    // float-float residual that meets tol is confirmed in float64.
    auto outer_residual = [&](int outer, bool ff) -> int {
        int s2 = outer == 0 ? source_and_residual<T>(H, B, lam, dt, r, rout)
                            : composite<T>(H, B, H->S, -1.0, -lamdt, 1.0, r, true, rout, ff);
        if (s2) return s2;
        int ef = 0;
        if ((s2 = read_norms(H, nr, &ef))) return s2;
        return ef ? OHM_ERR_INVALID : OHM_OK;
    };
    bool ff = false;
    for (int outer = 0;; outer++) {
        if ((st = outer_residual(outer, ff))) return st;
        if (ff && tol >= 0 && nr[0] <= tol && (st = outer_residual(outer, false))) return st;
        if (outer == 0) first = nr[0];
        if (!std::isfinite(nr[0]) || !std::isfinite(nr[1])) {
            result = OHM_ERR_NONFINITE;
            break;
        }
        if (tol >= 0 && nr[0] <= tol) break;
        if (cycles >= H->d.max_outer) {
            result = tol >= 0 ? OHM_ERR_NOT_CONVERGED : OHM_OK;
            break;
        }
        const double fl = inner_floor(H);
        const double target = tol >= 0 ? std::max(fl, 0.3 * tol / std::max(nr[0], 1e-300)) : fl;
        ff = H->ff_mid && !(tol >= 0 && nr[0] * target <= tol);
        if (H->d.krylov > 0) {
            if ((st = inner_fgmres<float>(H, lamdt, target, &cycles))) return st;
        } else {
        CK(cudaMemsetAsync(eacc, 0, nbytes, H->s));
        double prev = 1.0;
        int ef = 0;
        while (cycles < H->d.max_outer) {
            if ((st = vcycle<T>(H, lamdt))) return st;
            for (auto &g : H->amr)
                LAUNCH(H, OHM_K_UPDATE, g.n(), launch_axpy_leaf<T>(g.dev, amr_ptr<T>(eacc, g, 3), amr_ptr<T>(e, g, 3), nullptr, H->s));
            cycles++;
            if ((st = sync_down_t<T>(H, eacc))) return st;
            if ((st = fill_ghosts_t<T>(H, eacc, (T *)H->ghostE))) return st;
            if ((st = composite_t<T, T>(H, eacc, rout, (const T *)H->amrbuf.eta, (const T *)H->ghostE,
                                        (const T *)H->ghostEtaT, -1.0, -lamdt, 1.0, r, (T *)nullptr, true)))
                return st;
            double ni[4];
            if ((st = read_norms(H, ni, &ef))) return st;
            // stop at the target, or when a cycle gains less than 10% (float32 stagnation)
            if (!std::isfinite(ni[0]) || ni[0] <= target || ni[0] > 0.9 * prev) break;
            prev = ni[0];
        }
        }
        if ((st = update_all<T>(H, B, eacc))) return st;
        if ((st = sync_down(H, B))) return st;
        if ((st = fill_ghosts_B(H, B))) return st;
    }
    if (stats) {
        stats->cycles = cycles;
        stats->converged = (result == OHM_OK && tol >= 0) ? 1 : 0;
        stats->rel_l2_initial = first;
        stats->rel_l2 = nr[0];
        stats->max_abs = nr[1];
    }
    return result;
}

// ---------------------------------------------------------------- batches of instances
// Per-instance norms, enqueued by composite_t into dnormK, copied to the host with the error
// word; the caller synchronises (read_norms_batch) or the copies end a captured graph.
int enqueue_norm_copy(ohm_hier *H) {
    CK(cudaMemcpyAsync(H->hnormK, H->dnormK, (size_t)H->K * 4 * sizeof(double), cudaMemcpyDeviceToHost, H->s));
    CK(cudaMemcpyAsync(H->hnorm + 4, H->d_err, sizeof(int), cudaMemcpyDeviceToHost, H->s));
    return OHM_OK;
}

int read_norms_batch(ohm_hier *H, std::vector<double> &rel, std::vector<double> &mx, int *err_flag) {
    CK(cudaStreamSynchronize(H->s));
    rel.resize(H->K);
    mx.resize(H->K);
    for (int q = 0; q < H->K; q++) {
        const double sr = H->hnormK[4 * q], ss = H->hnormK[4 * q + 1];
        rel[q] = ss > 0 ? std::sqrt(sr / ss) : std::sqrt(sr);
        mx[q] = H->hnormK[4 * q + 2];
    }
    int e;
    memcpy(&e, &H->hnorm[4], sizeof(int));
    *err_flag = e;
    return OHM_OK;
}

// Runs `enqueue` (stream work only, no synchronisation) eagerly, or, with use_graphs on a
// non-default stream, replays a CUDA graph captured from it on its second use.
template <class F>
int run_iteration(ohm_hier *H, F enqueue) {
    const bool want = H->d.use_graphs && H->s != nullptr && !H->graph_failed && H->prof_kind < 0;
    if (!want) return enqueue();
    if (!H->graph) {
        if (!H->graph_warm) {  // first use eager: lazy per-kernel attributes are set outside capture
            H->graph_warm = true;
            return enqueue();
        }
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(H->s, cudaStreamCaptureModeThreadLocal));
        const int64_t n0 = H->nlaunch;
        const int st = enqueue();
        const cudaError_t ec = cudaStreamEndCapture(H->s, &g);
        cudaError_t ei = cudaErrorUnknown;
        if (st == OHM_OK && ec == cudaSuccess) ei = cudaGraphInstantiate(&H->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (st != OHM_OK || ec != cudaSuccess || ei != cudaSuccess) {
            cudaGetLastError();
            H->graph = nullptr;
            H->graph_failed = true;
            H->nlaunch = n0;
            return enqueue();  // nothing was executed by the capture: run eagerly
        }
        H->graph_launches = H->nlaunch - n0;
        H->nlaunch = n0;
    }
    H->nlaunch += H->graph_launches;
    CK(cudaGraphLaunch(H->graph, H->s));
    return OHM_OK;
}

// eta * dt[q] on every block of instance q, then the derived eta arrays
template <typename T>
int batch_scale(ohm_hier *H, const double *dt) {
    bool same = !H->eta_dirty && (int)H->cur_scale.size() == H->K;
    for (int q = 0; same && q < H->K; q++) same = H->cur_scale[q] == dt[q];
    if (same) return OHM_OK;
    std::vector<double> bs((size_t)H->nblocks);
    for (int l = 0; l < H->ranges.nlev; l++)
        for (int q = 0; q < H->K; q++)
            for (int b = 0; b < H->ranges.n[l]; b++) bs[(size_t)H->ranges.off[l] + (size_t)q * H->ranges.n[l] + b] = dt[q];
    CK(cudaMemcpyAsync(H->bscale, bs.data(), bs.size() * sizeof(double), cudaMemcpyHostToDevice, H->s));
    CK(cudaStreamSynchronize(H->s));
    CK(launch_scale_blocks(H->eta_user, H->eta64, H->bscale, (int)H->nblocks, H->s));
    int st;
    if ((st = eta_derive<T>(H))) return st;
    H->cur_scale.assign(dt, dt + H->K);
    H->eta_dirty = false;
    return OHM_OK;
}

// ---- batched FGMRES: one Arnoldi recurrence per instance, every launch covering the batch
// Per-instance products <w, v_i> (i < S.k) and <w, w> into kdots, left on the device; with
// gate, nothing runs unless the device flag is set.
int mdot_inst_dev(ohm_hier *H, const float *w, const VecSet &S, const int *gate = nullptr) {
    LAUNCH(H, OHM_K_KRYLOV, (int)H->nblocks,
           launch_mdot_inst(w, S, H->wblk, (int)H->nblocks, H->ranges, H->K, H->kpart, H->kdots, H->s, gate));
    return OHM_OK;
}

// dst = (src - sum_i coef[q][i] v_i) * coef[q][KMAX] with the coefficients on the device
int maxpy_inst_dev(ohm_hier *H, float *dst, const float *src, const VecSet &S, const int *gate = nullptr) {
    LAUNCH(H, OHM_K_KRYLOV, (int)H->nblocks,
           launch_maxpy_inst(dst, src, S, H->kcoef, H->binst, (size_t)H->nblocks * 3 * B3, H->s, gate));
    return OHM_OK;
}

#define FG(op, j) LAUNCH(H, OHM_K_KRYLOV, 0, launch_fg(H->fg, op, j, H->s))

// While a kernel kind is being timed (never under graph capture), the share of instances the
// device-side mask lets through is read back so that the timed launches count only the cells
// they iterate.
int fg_prof_mask(ohm_hier *H) {
    if (H->prof_kind < 0) return OHM_OK;
    char *hs = H->fg_host + (size_t)H->K * 13;
    CK(cudaMemcpyAsync(hs, H->fg.imask, H->K, cudaMemcpyDeviceToHost, H->s));
    CK(cudaStreamSynchronize(H->s));
    H->active_frac = (double)std::count_if(hs, hs + H->K, [](char v) { return v != 0; }) / H->K;
    return OHM_OK;
}

// One restart cycle of the batched FGMRES(m), stream work only: m Arnoldi steps (each: the V-cycle and the operator on the active instances, classical
// Gram-Schmidt with one-pass normalisation, or a measured norm where cancellation was large --
// that pass returns at once on the device when no instance needs it -- and the Givens update),
// the solution update x += Z y, then the true residual rhs - L x, its norm and the restart
// decisions; finally the live flags and cycle counts are copied to pinned host memory.
int fg_cycle(ohm_hier *H, double lamdt) {
    const int m = H->d.krylov;
    float *x = (float *)H->eacc, *rhs = (float *)H->rout;
    VecSet none;
    none.k = 0;
    int st;
    FG(FG_CYCLE, 0);
    for (int j = 0; j < m; j++) {
        FG(FG_ACT, j);
        if ((st = fg_prof_mask(H))) return st;
        void *r_save = H->amrbuf.r, *e_save = H->amrbuf.e;
        H->amrbuf.r = H->kv[j];
        H->amrbuf.e = H->kz[j];
        st = vcycle<float>(H, lamdt);
        H->amrbuf.r = r_save;
        H->amrbuf.e = e_save;
        if (st) return st;
        if ((st = apply_L32(H, H->kz[j], nullptr, 1.0, lamdt, 0.0, H->kv[j + 1], lamdt))) return st;
        VecSet S;
        S.k = j + 1;
        for (int i = 0; i <= j; i++) S.v[i] = H->kv[i];
        if ((st = mdot_inst_dev(H, H->kv[j + 1], S))) return st;
        FG(FG_ORTHO, j);
        // v_m, formed by the last step, is never read: that step orthogonalises only where a
        // norm must be measured, and scales nothing
        const bool last = j + 1 == m;
        if ((st = maxpy_inst_dev(H, H->kv[j + 1], H->kv[j + 1], S, last ? H->fg.any_need2 : nullptr))) return st;
        if ((st = mdot_inst_dev(H, H->kv[j + 1], none, H->fg.any_need2))) return st;
        FG(FG_RENORM, j);
        if (!last && (st = maxpy_inst_dev(H, H->kv[j + 1], H->kv[j + 1], none, H->fg.any_need2))) return st;
        FG(FG_GIVENS, j);
    }
    FG(FG_SOLVE, 0);
    VecSet Z;
    Z.k = m;
    for (int i = 0; i < m; i++) Z.v[i] = H->kz[i];
    if ((st = maxpy_inst_dev(H, x, x, Z))) return st;
    FG(FG_RESTART_MASK, 0);
    if ((st = fg_prof_mask(H))) return st;
    if ((st = apply_L32(H, x, rhs, -1.0, -lamdt, 1.0, H->kv[0], lamdt))) return st;
    if ((st = mdot_inst_dev(H, H->kv[0], none))) return st;
    FG(FG_RESTART, 0);
    if ((st = maxpy_inst_dev(H, H->kv[0], H->kv[0], none))) return st;
    const int K = H->K;
    CK(cudaMemcpyAsync(H->fg_host + (size_t)K * 12, H->fg.live, K, cudaMemcpyDeviceToHost, H->s));
    CK(cudaMemcpyAsync(H->fg_host + (size_t)K * 8, H->fg.cycles, (size_t)K * sizeof(int), cudaMemcpyDeviceToHost, H->s));
    return OHM_OK;
}

// Runs fg_cycle eagerly, or (use_graphs, non-default stream) replays a CUDA graph captured from
// it on its second use: every pointer, count and coefficient it needs lives on the device.
int run_fg_cycle(ohm_hier *H, double lamdt) {
    const bool want = H->d.use_graphs && H->s != nullptr && !H->fg_failed && H->prof_kind < 0;
    if (!want) return fg_cycle(H, lamdt);
    if (!H->fg_graph) {
        if (!H->fg_warm) {
            H->fg_warm = true;
            return fg_cycle(H, lamdt);
        }
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(H->s, cudaStreamCaptureModeThreadLocal));
        const int64_t n0 = H->nlaunch;
        const int st = fg_cycle(H, lamdt);
        const cudaError_t ec = cudaStreamEndCapture(H->s, &g);
        cudaError_t ei = cudaErrorUnknown;
        if (st == OHM_OK && ec == cudaSuccess) ei = cudaGraphInstantiate(&H->fg_graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (st != OHM_OK || ec != cudaSuccess || ei != cudaSuccess) {
            cudaGetLastError();
            H->fg_graph = nullptr;
            H->fg_failed = true;
            H->nlaunch = n0;
            return fg_cycle(H, lamdt);  // the capture executed nothing: run eagerly
        }
        H->fg_launches = H->nlaunch - n0;
        H->nlaunch = n0;
    }
    H->nlaunch += H->fg_launches;
    CK(cudaGraphLaunch(H->fg_graph, H->s));
    return OHM_OK;
}

// Float32 inner solve of L x = rout for every instance q with run[q], by FGMRES(m) right-
// preconditioned by one V-cycle, as inner_fgmres does for one problem: each instance has its
// own Arnoldi basis coefficients, Hessenberg matrix, Givens rotations, restarts and stopping
// test (target[q], stagnation, V-cycle budget), so its iterates do not depend on the others;
// the V-cycles, operator applications and vector kernels of all running instances share
// launches, and instances that stopped are skipped by the compute mask.  The scalar recurrence
// runs on the device (k_fg), so the host waits once per restart cycle.  x is left in eacc.
int inner_fgmres_batch(ohm_hier *H, double lamdt, const std::vector<double> &target, const uint8_t *run,
                       std::vector<int> &cycles) {
    const int K = H->K;
    const size_t nel = (size_t)H->nblocks * 3 * B3;
    float *x = (float *)H->eacc, *rhs = (float *)H->rout;
    int st;
    // target (doubles), cycles (ints) and run flags in, through the pinned staging area
    char *hs = H->fg_host;
    memcpy(hs, target.data(), (size_t)K * sizeof(double));
    memcpy(hs + (size_t)K * 8, cycles.data(), (size_t)K * sizeof(int));
    memcpy(hs + (size_t)K * 12, run, K);
    CK(cudaMemcpyAsync(H->fg.target, hs, (size_t)K * sizeof(double), cudaMemcpyHostToDevice, H->s));
    CK(cudaMemcpyAsync(H->fg.cycles, hs + (size_t)K * 8, (size_t)K * sizeof(int), cudaMemcpyHostToDevice, H->s));
    CK(cudaMemcpyAsync(H->fg.run, hs + (size_t)K * 12, K, cudaMemcpyHostToDevice, H->s));
    CK(cudaMemsetAsync(x, 0, nel * sizeof(float), H->s));
    VecSet none;
    none.k = 0;
    if ((st = mdot_inst_dev(H, rhs, none))) return st;
    FG(FG_START, 0);
    if ((st = maxpy_inst_dev(H, H->kv[0], rhs, none))) return st;
    CK(cudaMemcpyAsync(hs + (size_t)K * 12, H->fg.live, K, cudaMemcpyDeviceToHost, H->s));
    CK(cudaStreamSynchronize(H->s));  // the staging area is read back below and reused
    H->cmask = H->fg.imask;
    H->active_frac = 1.0;
    bool any = std::any_of(hs + (size_t)K * 12, hs + (size_t)K * 13, [](char v) { return v != 0; });
    while (any) {
        st = run_fg_cycle(H, lamdt);
        if (st) break;
        if (cudaStreamSynchronize(H->s) != cudaSuccess) {
            st = OHM_ERR_CUDA;
            break;
        }
        any = std::any_of(hs + (size_t)K * 12, hs + (size_t)K * 13, [](char v) { return v != 0; });
    }
    H->cmask = nullptr;
    if (st) return st;
    memcpy(cycles.data(), hs + (size_t)K * 8, (size_t)K * sizeof(int));
    return OHM_OK;
}

// Batched theta step (dt folded into eta per instance, so the operator's lambda dt is lambda):
// the outer float64 loop of Eqs. 16-18 per instance, with a float32 defect-correction inner
// solve (mixed) or one float64 V-cycle per outer iteration (FP64).  Instances are stopped and
// masked out one by one; every launch covers the whole batch.
template <typename T>
int cn_step_batch_t(ohm_hier *H, double *B, const double *dt, double tol, const uint8_t *active,
                    ohm_step_stats *stats) {
    const int K = H->K;
    const double lam = H->d.lambda, lamdt = lam;
    int st;
    if ((st = batch_scale<T>(H, dt))) return st;
    if ((st = prepare_dt<T>(H, 1.0))) return st;
    CK(cudaMemsetAsync(H->d_err, 0, sizeof(int), H->s));
    if ((st = sync_down(H, B))) return st;
    if ((st = fill_ghosts_B(H, B))) return st;
    H->has_S = true;
    H->last_dt = 1.0;
    enum { RUN = 0, DONE = 1, NOCONV = 2, NONFIN = 3, IDLE = 4 };
    std::vector<int> state(K), cycles(K, 0);
    std::vector<double> first(K, 0.0), rel, mx, ni, nmx, target(K), prev(K);
    for (int q = 0; q < K; q++) state[q] = (active && !active[q]) ? IDLE : RUN;
    uint8_t *omask_h = H->imask_h, *imask_h = H->imask_h + K;
    uint8_t *omask_d = H->imask_d, *imask_d = H->imask_d + K;
    T *r = (T *)H->amrbuf.r, *e = (T *)H->amrbuf.e;
    T *rout = (T *)H->rout, *eacc = (T *)H->eacc;
    const size_t nbytes = (size_t)H->nblocks * 3 * B3 * sizeof(T);
    const double fl = inner_floor(H);
    for (int outer = 0;; outer++) {
        T *r2 = H->mixed ? rout : (T *)nullptr;
        if ((st = outer == 0 ? source_and_residual<T>(H, B, lam, 1.0, r, r2)
                             : composite<T>(H, B, H->S, -1.0, -lamdt, 1.0, r, true, r2)))
            return st;
        if ((st = enqueue_norm_copy(H))) return st;
        int ef = 0;
        if ((st = read_norms_batch(H, rel, mx, &ef))) return st;
        if (ef) return OHM_ERR_INVALID;
        bool any = false;
        for (int q = 0; q < K; q++) {
            omask_h[q] = 0;
            if (state[q] != RUN) continue;
            if (outer == 0) first[q] = rel[q];
            if (!std::isfinite(rel[q]) || !std::isfinite(mx[q])) state[q] = NONFIN;
            else if (tol >= 0 && rel[q] <= tol) state[q] = DONE;
            else if (cycles[q] >= H->d.max_outer) state[q] = tol >= 0 ? NOCONV : DONE;
            else {
                omask_h[q] = 1;
                any = true;
            }
        }
        if (!any) break;
        CK(cudaMemcpyAsync(omask_d, omask_h, K, cudaMemcpyHostToDevice, H->s));
        if (!H->mixed) {
            // one float64 V-cycle for every running instance (the others' blocks are skipped)
            H->cmask = omask_d;
            H->active_frac = (double)std::count(omask_h, omask_h + K, 1) / K;
            st = vcycle<T>(H, lamdt);
            H->cmask = nullptr;
            if (st) return st;
            if ((st = update_all<T>(H, B, e, omask_d))) return st;
            for (int q = 0; q < K; q++) cycles[q] += omask_h[q];
        } else {
            CK(cudaMemsetAsync(eacc, 0, nbytes, H->s));
            for (int q = 0; q < K; q++) {
                imask_h[q] = omask_h[q];
                target[q] = tol >= 0 ? std::max(fl, 0.3 * tol / std::max(rel[q], 1e-300)) : fl;
                prev[q] = 1.0;
            }
            bool inner = true;
            if (H->d.krylov > 0) {  // per-instance FGMRES instead of defect correction
                if constexpr (std::is_same<T, float>::value) {
                    if ((st = inner_fgmres_batch(H, lamdt, target, omask_h, cycles))) return st;
                }
                inner = false;
            }
            while (inner) {
                CK(cudaMemcpyAsync(imask_d, imask_h, K, cudaMemcpyHostToDevice, H->s));
                H->cmask = imask_d;  // blocks of instances that stopped iterating are skipped
                H->active_frac = (double)std::count(imask_h, imask_h + K, 1) / K;
                st = run_iteration(H, [&]() -> int {
                    int s2;
                    if ((s2 = vcycle<T>(H, lamdt))) return s2;
                    for (auto &g : H->amr)
                        LAUNCH(H, OHM_K_UPDATE, g.n(), launch_axpy_leaf<T>(g.dev, amr_ptr<T>(eacc, g, 3), amr_ptr<T>(e, g, 3), imask_d, H->s));
                    if ((s2 = sync_down_t<T>(H, eacc))) return s2;
                    if ((s2 = fill_ghosts_t<T>(H, eacc, (T *)H->ghostE))) return s2;
                    if ((s2 = composite_t<T, T>(H, eacc, rout, (const T *)H->amrbuf.eta, (const T *)H->ghostE,
                                                (const T *)H->ghostEtaT, -1.0, -lamdt, 1.0, r, (T *)nullptr, true)))
                        return s2;
                    return enqueue_norm_copy(H);
                });
                H->cmask = nullptr;
                if (st) return st;
                if ((st = read_norms_batch(H, ni, nmx, &ef))) return st;
                inner = false;
                for (int q = 0; q < K; q++) {
                    if (!imask_h[q]) continue;
                    cycles[q]++;
                    // stop at the target, on float32 stagnation (< 10% gained) or at the budget
                    if (!std::isfinite(ni[q]) || ni[q] <= target[q] || ni[q] > 0.9 * prev[q] || cycles[q] >= H->d.max_outer)
                        imask_h[q] = 0;
                    else {
                        prev[q] = ni[q];
                        inner = true;
                    }
                }
            }
            if ((st = update_all<T>(H, B, eacc, omask_d))) return st;
        }
        if ((st = sync_down(H, B))) return st;
        if ((st = fill_ghosts_B(H, B))) return st;
    }
    int result = OHM_OK;
    for (int q = 0; q < K; q++) {
        if (state[q] == NONFIN) result = OHM_ERR_NONFINITE;
        else if (state[q] == NOCONV && result == OHM_OK) result = OHM_ERR_NOT_CONVERGED;
        if (!stats) continue;
        ohm_step_stats &o = stats[q];
        memset(&o, 0, sizeof(o));
        if (state[q] == IDLE) continue;
        o.cycles = cycles[q];
        o.converged = (state[q] == DONE && tol >= 0) ? 1 : 0;
        o.rel_l2_initial = first[q];
        o.rel_l2 = rel[q];
        o.max_abs = mx[q];
    }
    return result;
}

bool valid_desc(const ohm_hier_desc *d, std::string &err) {
    if (!d) { err = "NULL descriptor"; return false; }
    for (int a = 0; a < 3; a++)
        if (d->base_cells[a] <= 0 || d->base_cells[a] % BS) { err = "base cells must be positive multiples of 8"; return false; }
    if (!(d->dx0 > 0) || !std::isfinite(d->dx0)) { err = "dx0 must be positive"; return false; }
    if (d->nlevels < 1 || d->nlevels > MAX_LEVELS) { err = "nlevels out of range"; return false; }
    if (d->nblocks <= 0 || !d->block_lijk) { err = "empty block list"; return false; }
    if (!(d->lambda > 0 && d->lambda <= 1)) { err = "lambda must be in (0, 1]"; return false; }
    if (d->precision != OHM_FP64 && d->precision != OHM_MIXED && d->precision != OHM_MIXED_FF &&
        d->precision != OHM_MIXED_FF_CHECKED) {
        err = "unknown precision";
        return false;
    }
    if (d->nu_pre < 0 || d->nu_post < 0 || d->n_coarse < 1 || d->max_outer < 1) { err = "bad cycle counts"; return false; }
    if (!(d->omega == 0 || (d->omega > 0 && d->omega < 2))) { err = "omega must be 0 (= 1) or in (0, 2)"; return false; }
    if (d->nu_coarse_pre < 0 || d->nu_coarse_post < 0) { err = "bad coarse-grid sweep counts"; return false; }
    if (d->krylov < 0 || d->krylov >= KMAX || (d->krylov > 0 && d->precision == OHM_FP64 && d->n_instances >= 1)) {
        err = "krylov must be 0, or 1..11 (batched hierarchies: with mixed precision only)";
        return false;
    }
    if (!(d->inner_tol >= 0 && d->inner_tol < 1)) { err = "inner_tol must be in [0, 1)"; return false; }
    if (d->n_instances < 0 || d->n_instances > (1 << 16)) { err = "n_instances out of range"; return false; }
    if ((int64_t)std::max(1, d->n_instances) * d->nblocks >= (int64_t)1 << 31) { err = "too many blocks"; return false; }
    for (int a = 0; a < 3; a++)
        if (((int64_t)d->base_cells[a] << (d->nlevels - 1)) >= (1 << 20)) { err = "level too fine"; return false; }
    return true;
}

thread_local std::string g_last_error;

}  // namespace

// ============================================================================ C ABI
extern "C" {

const char *ohm_status_string(int status) {
    switch (status) {
        case OHM_OK: return "ok";
        case OHM_ERR_INVALID: return g_last_error.empty() ? "invalid argument" : g_last_error.c_str();
        case OHM_ERR_NOT_CONVERGED: return "not converged within max_outer cycles";
        case OHM_ERR_NONFINITE: return "residual became non-finite";
        case OHM_ERR_OOM: return "device allocation failed";
        case OHM_ERR_CUDA: return "CUDA error";
        case -6: return "timed out (ohm_server_wait)";
        default: return "unknown status";
    }
}

int ohm_create_hierarchy(const ohm_hier_desc *d, ohm_hier **out) {
    if (!out) return OHM_ERR_INVALID;
    *out = nullptr;
    std::string err;
    if (!valid_desc(d, err)) {
        g_last_error = err;
        return OHM_ERR_INVALID;
    }
    ohm_hier *H = new ohm_hier();
    H->d = *d;
    if (H->d.omega == 0) H->d.omega = 1.0;
    H->d.block_lijk = nullptr;
    H->s = (cudaStream_t)d->stream;
    H->mixed = d->precision != OHM_FP64;
    H->ff = d->precision == OHM_MIXED_FF;
    H->ff_mid = d->precision == OHM_MIXED_FF_CHECKED;
    H->nlev = d->nlevels;
    H->nblocks = d->nblocks;
    H->lijk.assign(d->block_lijk, d->block_lijk + 4 * d->nblocks);
    H->batched = d->n_instances >= 1;
    H->K = std::max(1, d->n_instances);
    H->nblk_inst = d->nblocks;
    int st = build_tables(H, err);
    if (st == OHM_OK && H->batched) replicate(H);
    if (st == OHM_OK) st = allocate(H, err);
    if (st != OHM_OK) {
        g_last_error = err;
        ohm_destroy(H);
        return st;
    }
    *out = H;
    return OHM_OK;
}

int ohm_hierarchy_bytes(const ohm_hier_desc *d, int64_t *bytes) {
    std::string err;
    if (!bytes || !valid_desc(d, err)) {
        g_last_error = bytes ? err : "NULL output";
        return OHM_ERR_INVALID;
    }
    ohm_hier H;
    H.d = *d;
    H.d.block_lijk = nullptr;
    H.mixed = d->precision != OHM_FP64;
    H.ff = d->precision == OHM_MIXED_FF;
    H.ff_mid = d->precision == OHM_MIXED_FF_CHECKED;
    H.nlev = d->nlevels;
    H.nblocks = d->nblocks;
    H.lijk.assign(d->block_lijk, d->block_lijk + 4 * d->nblocks);
    H.batched = d->n_instances >= 1;
    H.K = std::max(1, d->n_instances);
    H.nblk_inst = d->nblocks;
    int st = build_tables(&H, err);
    if (st == OHM_OK && H.batched) replicate(&H);
    if (st == OHM_OK) st = allocate(&H, err, bytes);
    if (st != OHM_OK) g_last_error = err;
    return st;
}

void ohm_destroy(ohm_hier *h) {
    if (!h) return;
    for (auto ev : h->prof_ev) cudaEventDestroy(ev);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->fg_graph) cudaGraphExecDestroy(h->fg_graph);
    if (h->pool) cudaFree(h->pool);
    if (h->fg_host) cudaFreeHost(h->fg_host);
    if (h->hnorm) cudaFreeHost(h->hnorm);
    if (h->hnormK) cudaFreeHost(h->hnormK);
    if (h->imask_h) cudaFreeHost(h->imask_h);
    delete h;
}

int ohm_set_eta(ohm_hier *h, const double *eta_dev) {
    if (!h || !eta_dev) return OHM_ERR_INVALID;
    if (h->batched) {  // scaled by each instance's dt at the next step
        CK(cudaMemcpyAsync(h->eta_user, eta_dev, (size_t)h->nblocks * B3 * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
        h->eta_dirty = true;
        h->eta_set = true;
        return OHM_OK;
    }
    if (h->eta_set) {
        // the same values again (a time loop passing its eta every step): the coarse levels,
        // ghosts and inverse diagonals derived from them are still valid.  The comparison
        // writes its flag straight into pinned host memory (device-accessible under unified
        // addressing), so reading it waits only for this stream, never for a copy engine that
        // another stream keeps busy with a large transfer.
        volatile int *flag = reinterpret_cast<volatile int *>(h->hnorm + 24);
        *flag = 0;  // no earlier comparison is in flight: each is waited for before its call returns
        if (h->flag_dev) {
            CK(launch_differs(eta_dev, h->eta64, (size_t)h->nblocks * B3, h->flag_dev, h->s));
        } else {  // pinned memory not mapped into the device: copy the flag back
            int *dflag = (int *)(h->dnorm + 6);
            CK(cudaMemsetAsync(dflag, 0, sizeof(int), h->s));
            CK(launch_differs(eta_dev, h->eta64, (size_t)h->nblocks * B3, dflag, h->s));
            CK(cudaMemcpyAsync((void *)flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, h->s));
        }
        CK(cudaStreamSynchronize(h->s));
        if (!*flag) return OHM_OK;
    }
    CK(cudaMemcpyAsync(h->eta64, eta_dev, (size_t)h->nblocks * B3 * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
    int st = h->mixed ? eta_derive<float>(h) : eta_derive<double>(h);
    if (st) return st;
    h->eta_set = true;
    return OHM_OK;
}

int ohm_cn_step_batch(ohm_hier *h, double *B_dev, const double *dt, double tol, const uint8_t *active,
                      ohm_step_stats *stats) {
    if (!h || !h->batched || !B_dev || !dt || !h->eta_set) return OHM_ERR_INVALID;
    for (int q = 0; q < h->K; q++)
        if ((!active || active[q]) && !(dt[q] > 0 && std::isfinite(dt[q]))) return OHM_ERR_INVALID;
    // inactive instances keep the scale they had (any positive value)
    std::vector<double> dts(dt, dt + h->K);
    for (int q = 0; q < h->K; q++)
        if (!(dts[q] > 0 && std::isfinite(dts[q]))) dts[q] = (int)h->cur_scale.size() == h->K ? h->cur_scale[q] : 1.0;
    return h->mixed ? cn_step_batch_t<float>(h, B_dev, dts.data(), tol, active, stats)
                    : cn_step_batch_t<double>(h, B_dev, dts.data(), tol, active, stats);
}

static void reset_graph(ohm_hier *h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_warm = false;
    if (h->fg_graph) cudaGraphExecDestroy(h->fg_graph);
    h->fg_graph = nullptr;
    h->fg_warm = false;
    h->fg.max_outer = h->d.max_outer;
}

int ohm_autotune(ohm_hier *h, const double *B_dev, const double *dt, double tol, ohm_tune_result *res) {
    if (!h || !B_dev || !dt || !h->eta_set) return OHM_ERR_INVALID;
    const size_t bytes = (size_t)h->nblocks * 3 * B3 * sizeof(double);
    double *Bw = nullptr;
    if (cudaMalloc(&Bw, bytes) != cudaSuccess) {
        cudaGetLastError();
        return OHM_ERR_OOM;
    }
    cudaEvent_t ev[2];
    cudaEventCreate(&ev[0]);
    cudaEventCreate(&ev[1]);
    const ohm_hier_desc saved = h->d;
    const int saved_sm = h->smoother;
    auto step = [&]() -> int {
        if (cudaMemcpyAsync(Bw, B_dev, bytes, cudaMemcpyDeviceToDevice, h->s) != cudaSuccess) return OHM_ERR_CUDA;
        if (h->batched) return ohm_cn_step_batch(h, Bw, dt, tol, nullptr, nullptr);
        return h->mixed ? cn_step_mixed(h, Bw, dt[0], tol, nullptr) : cn_step_impl<double>(h, Bw, dt[0], tol, nullptr);
    };
    int st = step();  // warm-up: first-use setup outside the timings
    const int nus[6][2] = {{1, 1}, {2, 1}, {2, 2}, {3, 2}, {3, 3}, {4, 4}};
    const int ncs[2] = {4, 16};
    double best = INFINITY;
    ohm_tune_result br{};
    int ncand = 0;
    for (int a = 0; a < 6 && st != OHM_ERR_CUDA && (st == OHM_OK || st == OHM_ERR_NOT_CONVERGED); a++)
        for (int c = 0; c < 2 && st != OHM_ERR_CUDA; c++)
            for (int sm = 0; sm < (h->mixed ? 2 : 1) && st != OHM_ERR_CUDA; sm++) {
                h->d.nu_pre = nus[a][0];
                h->d.nu_post = nus[a][1];
                h->d.n_coarse = ncs[c];
                h->smoother = h->mixed ? sm : 1;
                reset_graph(h);
                cudaEventRecord(ev[0], h->s);
                const int r = step();
                cudaEventRecord(ev[1], h->s);
                if (cudaEventSynchronize(ev[1]) != cudaSuccess) {
                    st = OHM_ERR_CUDA;
                    break;
                }
                ncand++;
                float ms = 0;
                cudaEventElapsedTime(&ms, ev[0], ev[1]);
                if (r == OHM_OK && ms < best) {
                    best = ms;
                    br = ohm_tune_result{h->d.nu_pre, h->d.nu_post, h->d.n_coarse, h->smoother, ms, 0, h->d.omega,
                                         h->d.nu_coarse_pre, h->d.nu_coarse_post};
                }
            }
    if ((st != OHM_OK && st != OHM_ERR_NOT_CONVERGED) || !(best < INFINITY)) {
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        cudaFree(Bw);
        h->d = saved;  // a failure, or nothing converged: keep the schedule the hierarchy had
        h->smoother = saved_sm;
        h->inv_dt = NAN;
        reset_graph(h);
        return st != OHM_OK && st != OHM_ERR_NOT_CONVERGED ? st : OHM_ERR_NOT_CONVERGED;
    }
    h->d.nu_pre = br.nu_pre;
    h->d.nu_post = br.nu_post;
    h->d.n_coarse = br.n_coarse;
    h->smoother = br.smoother;
    // V(1,1) and V(1,0) on the grids coarser than level 0, on the chosen schedule
    br.nu_coarse_pre = saved.nu_coarse_pre;
    br.nu_coarse_post = saved.nu_coarse_post;
    const int cnu[2][2] = {{1, 1}, {1, 0}};
    for (int q = 0; q < 2 && st != OHM_ERR_CUDA; q++) {
        if (saved.nu_coarse_pre == cnu[q][0] && saved.nu_coarse_post == cnu[q][1]) continue;
        h->d.nu_coarse_pre = cnu[q][0];
        h->d.nu_coarse_post = cnu[q][1];
        reset_graph(h);
        cudaEventRecord(ev[0], h->s);
        const int r = step();
        cudaEventRecord(ev[1], h->s);
        if (cudaEventSynchronize(ev[1]) != cudaSuccess) {
            st = OHM_ERR_CUDA;
            break;
        }
        ncand++;
        float ms = 0;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (r == OHM_OK && ms < best) {
            best = ms;
            br.ms = ms;
            br.nu_coarse_pre = cnu[q][0];
            br.nu_coarse_post = cnu[q][1];
        }
    }
    h->d.nu_coarse_pre = br.nu_coarse_pre;
    h->d.nu_coarse_post = br.nu_coarse_post;
    // relaxation factor of the sweeps on the chosen schedule (folded into the inverse diagonals,
    // so they are recomputed for each candidate)
    br.omega = saved.omega;
    const double oms[4] = {1.0, 1.15, 1.3, 1.45};
    for (int q = 0; q < 4 && st != OHM_ERR_CUDA; q++) {
        if (oms[q] == saved.omega) continue;
        h->d.omega = oms[q];
        h->inv_dt = NAN;
        reset_graph(h);
        cudaEventRecord(ev[0], h->s);
        const int r = step();
        cudaEventRecord(ev[1], h->s);
        if (cudaEventSynchronize(ev[1]) != cudaSuccess) {
            st = OHM_ERR_CUDA;
            break;
        }
        ncand++;
        float ms = 0;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (r == OHM_OK && ms < best) {
            best = ms;
            br.ms = ms;
            br.omega = oms[q];
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    cudaFree(Bw);
    h->d.omega = br.omega;
    h->inv_dt = NAN;
    reset_graph(h);
    if (st == OHM_ERR_CUDA) {
        h->d = saved;
        h->smoother = saved_sm;
        return st;
    }
    br.candidates = ncand;
    if (res) *res = br;
    return OHM_OK;
}

int ohm_cn_step(ohm_hier *h, double *B_dev, const double *eta_dev, double dt, double tol, ohm_step_stats *stats) {
    if (!h || h->batched || !B_dev || !(dt > 0) || !std::isfinite(dt)) return OHM_ERR_INVALID;
    if (eta_dev) {
        int st = ohm_set_eta(h, eta_dev);
        if (st) return st;
    }
    if (!h->eta_set) return OHM_ERR_INVALID;
    return h->mixed ? cn_step_mixed(h, B_dev, dt, tol, stats) : cn_step_impl<double>(h, B_dev, dt, tol, stats);
}

int ohm_residual_norm(ohm_hier *h, const double *B_dev, double *rel_l2, double *max_abs) {
    if (!h || h->batched || !B_dev || !h->has_S || !h->eta_set) return OHM_ERR_INVALID;
    CK(cudaMemcpyAsync(h->Bscr, B_dev, (size_t)h->nblocks * 3 * B3 * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
    int st;
    CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->s));
    if ((st = sync_down(h, h->Bscr))) return st;
    if ((st = fill_ghosts_B(h, h->Bscr))) return st;
    // the residual itself lands in the multigrid right-hand side buffer (not needed further)
    int st2 = h->mixed ? composite<float>(h, h->Bscr, h->S, -1.0, -h->d.lambda * h->last_dt, 1.0, (float *)h->amrbuf.r, true)
                       : composite<double>(h, h->Bscr, h->S, -1.0, -h->d.lambda * h->last_dt, 1.0, (double *)h->amrbuf.r, true);
    if (st2) return st2;
    double nr[4];
    int ef = 0;
    if ((st = read_norms(h, nr, &ef))) return st;
    if (rel_l2) *rel_l2 = nr[0];
    if (max_abs) *max_abs = nr[1];
    return ef ? OHM_ERR_INVALID : OHM_OK;
}

int ohm_op_sync_down(ohm_hier *h, double *B_dev) {
    if (!h || h->batched || !B_dev) return OHM_ERR_INVALID;
    return sync_down(h, B_dev);
}

static int op_composite(ohm_hier *h, const double *X, const double *Y, double a, double c, double d, double *out,
                        double *norms) {
    if (!h->eta_set) return OHM_ERR_INVALID;
    CK(cudaMemcpyAsync(h->Bscr, X, (size_t)h->nblocks * 3 * B3 * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
    CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->s));
    int st;
    if ((st = sync_down(h, h->Bscr))) return st;
    if ((st = fill_ghosts_B(h, h->Bscr))) return st;
    if ((st = composite<double>(h, h->Bscr, Y, a, c, d, out, norms != nullptr))) return st;
    for (auto &g : h->amr) CK(launch_zero_covered(g.dev, out + (size_t)g.off * 3 * B3, h->s));
    int ef = 0;
    if (norms) {
        if ((st = read_norms(h, norms, &ef))) return st;
    } else if ((st = read_err(h, &ef))) {
        return st;
    }
    return ef ? OHM_ERR_INVALID : OHM_OK;
}

int ohm_op_div_flux(ohm_hier *h, const double *B_dev, double *out_dev) {
    if (!h || h->batched || !B_dev || !out_dev) return OHM_ERR_INVALID;
    return op_composite(h, B_dev, nullptr, 0.0, 1.0, 0.0, out_dev, nullptr);
}

int ohm_op_source(ohm_hier *h, const double *b_dev, double dt, double *S_dev) {
    if (!h || h->batched || !b_dev || !S_dev || !(dt > 0)) return OHM_ERR_INVALID;
    return op_composite(h, b_dev, nullptr, 1.0, -(1.0 - h->d.lambda) * dt, 0.0, S_dev, nullptr);
}

int ohm_op_residual(ohm_hier *h, const double *B_dev, const double *S_dev, double dt, double *R_dev, double *norms) {
    if (!h || h->batched || !B_dev || !S_dev || !R_dev || !(dt > 0)) return OHM_ERR_INVALID;
    double tmp[4];
    return op_composite(h, B_dev, S_dev, -1.0, -h->d.lambda * dt, 1.0, R_dev, norms ? norms : tmp);
}

int ohm_op_vcycle(ohm_hier *h, const double *R_dev, double dt, double *e_dev) {
    if (!h || h->batched || !R_dev || !e_dev || !(dt > 0) || h->mixed || !h->eta_set) return OHM_ERR_INVALID;
    int st;
    if ((st = prepare_dt<double>(h, dt))) return st;
    CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->s));
    CK(cudaMemcpyAsync(h->amrbuf.r, R_dev, (size_t)h->nblocks * 3 * B3 * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
    if ((st = vcycle<double>(h, h->d.lambda * dt))) return st;
    CK(cudaMemcpyAsync(e_dev, h->amrbuf.e, (size_t)h->nblocks * 3 * B3 * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
    for (auto &g : h->amr) CK(launch_zero_covered(g.dev, e_dev + (size_t)g.off * 3 * B3, h->s));
    int ef = 0;
    if ((st = read_err(h, &ef))) return st;
    return ef ? OHM_ERR_INVALID : OHM_OK;
}

int ohm_prof_enable(ohm_hier *h, int kernel, int min_blocks, int max_launches) {
    if (!h || max_launches < 0 || max_launches > (1 << 20)) return OHM_ERR_INVALID;
    h->prof_kind = -1;
    for (auto ev : h->prof_ev) cudaEventDestroy(ev);
    h->prof_ev.clear();
    h->prof_used = 0;
    h->prof_launches = 0;
    h->prof_cells = 0;
    if (kernel < 0) return OHM_OK;
    h->prof_ev.resize(2 * (size_t)max_launches);
    for (auto &ev : h->prof_ev) CK(cudaEventCreate(&ev));
    h->prof_kind = kernel;
    h->prof_min_blocks = min_blocks;
    return OHM_OK;
}

int ohm_prof_read(ohm_hier *h, double *total_ms, int64_t *launches, int64_t *cells) {
    if (!h) return OHM_ERR_INVALID;
    CK(cudaStreamSynchronize(h->s));
    double tot = 0;
    for (int i = 0; i + 1 < h->prof_used; i += 2) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, h->prof_ev[i], h->prof_ev[i + 1]));
        tot += ms;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = h->prof_launches;
    if (cells) *cells = h->prof_cells;
    h->prof_used = 0;
    h->prof_launches = 0;
    h->prof_cells = 0;
    return OHM_OK;
}

int64_t ohm_launch_count(const ohm_hier *h) { return h ? h->nlaunch : -1; }

int ohm_mg_grid_info(ohm_hier *h, int m, int32_t dims[3], int64_t *nblocks, int32_t *ijk) {
    if (!h || m < 0) return OHM_ERR_INVALID;
    const int nmg = 1 + (int)h->mg.size() + (int)h->small.size();
    if (m >= nmg) return OHM_ERR_INVALID;
    if (m <= (int)h->mg.size()) {
        const HGrid &g = m == 0 ? h->amr[0] : h->mg[m - 1];
        if (dims) for (int a = 0; a < 3; a++) dims[a] = g.dims[a];
        if (nblocks) *nblocks = g.n();
        if (ijk) memcpy(ijk, g.bijk.data(), g.bijk.size() * sizeof(int32_t));
    } else {
        const auto &q = h->small[m - 1 - h->mg.size()];
        if (dims) for (int a = 0; a < 3; a++) dims[a] = q[a];
        if (nblocks) *nblocks = 0;
    }
    return OHM_OK;
}

// Single-grid steps: copy the caller's arrays into grid m's buffers, run one kernel, copy
// back.  They overwrite that grid's eta, so ohm_set_eta is required again before a step.
static int grid_setup(ohm_hier *h, int m, const double *eta_dev, double dt, GridRef &G) {
    if (!h || h->batched || h->mixed || m < 0 || m > (int)h->mg.size() || !eta_dev || !(dt > 0)) return OHM_ERR_INVALID;
    if (m == 0 && h->nlev > 1) return OHM_ERR_INVALID;
    G = base_ref<double>(h, m);
    const size_t nb = (size_t)G.g->n();
    CK(cudaMemcpyAsync(G.eta, eta_dev, nb * B3 * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
    // omega / (1 + alpha): the colour pass applies the hierarchy's relaxation factor
    CK(launch_invdiag<double>(gdev(h, *G.g), (const double *)G.eta, nullptr, h->d.lambda * dt, (double *)G.inv, h->s));
    h->eta_set = false;
    h->inv_dt = NAN;
    return OHM_OK;
}

int ohm_op_grid_smooth(ohm_hier *h, int m, double *e_dev, const double *r_dev, const double *eta_dev, double dt, int colour) {
    if (!e_dev || !r_dev || (colour != 0 && colour != 1)) return OHM_ERR_INVALID;
    GridRef G;
    int st;
    if ((st = grid_setup(h, m, eta_dev, dt, G))) return st;
    const size_t bytes = (size_t)G.g->n() * 3 * B3 * sizeof(double);
    CK(cudaMemcpyAsync(G.e, e_dev, bytes, cudaMemcpyDeviceToDevice, h->s));
    CK(cudaMemcpyAsync(G.r, r_dev, bytes, cudaMemcpyDeviceToDevice, h->s));
    CK(launch_smooth<double>(G.g->dev, (const double *)G.e, (double *)G.e2, (const double *)G.r, (const double *)G.eta,
                             (const double *)G.inv, nullptr, nullptr, h->d.lambda * dt, colour, h->s));
    CK(cudaMemcpyAsync(e_dev, G.e2, bytes, cudaMemcpyDeviceToDevice, h->s));
    CK(cudaStreamSynchronize(h->s));
    return OHM_OK;
}

int ohm_op_grid_residual(ohm_hier *h, int m, const double *e_dev, const double *r_dev, const double *eta_dev, double dt,
                         double *t_dev) {
    if (!e_dev || !r_dev || !t_dev) return OHM_ERR_INVALID;
    GridRef G;
    int st;
    if ((st = grid_setup(h, m, eta_dev, dt, G))) return st;
    const size_t bytes = (size_t)G.g->n() * 3 * B3 * sizeof(double);
    CK(cudaMemcpyAsync(G.e, e_dev, bytes, cudaMemcpyDeviceToDevice, h->s));
    CK(cudaMemcpyAsync(G.r, r_dev, bytes, cudaMemcpyDeviceToDevice, h->s));
    CK(launch_resid_restrict<double>(G.g->dev, (const double *)G.e, (const double *)G.r, (const double *)G.eta, nullptr,
                                     nullptr, h->d.lambda * dt, t_dev, nullptr, nullptr, nullptr, h->s));
    CK(cudaStreamSynchronize(h->s));
    return OHM_OK;
}

int ohm_op_grid_restrict(ohm_hier *h, int m, const double *fine_dev, double *coarse_dev, int ncomp) {
    if (!h || h->batched || h->mixed || !fine_dev || !coarse_dev || (ncomp != 1 && ncomp != 3)) return OHM_ERR_INVALID;
    if (m < 0 || m >= (int)h->mg.size() || (m == 0 && h->nlev > 1)) return OHM_ERR_INVALID;
    const HGrid &g = m == 0 ? h->amr[0] : h->mg[m - 1];
    CK(launch_restrict<double>(g.dev, fine_dev, ncomp, coarse_dev, nullptr, nullptr, h->s));
    CK(cudaStreamSynchronize(h->s));
    return OHM_OK;
}

int ohm_op_grid_prolong_add(ohm_hier *h, int m, const double *coarse_dev, double *fine_dev) {
    if (!h || h->batched || h->mixed || !fine_dev || !coarse_dev) return OHM_ERR_INVALID;
    if (m < 0 || m >= (int)h->mg.size() || (m == 0 && h->nlev > 1)) return OHM_ERR_INVALID;
    const HGrid &g = m == 0 ? h->amr[0] : h->mg[m - 1];
    CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->s));
    CK(launch_prolong_add<double>(g.dev, &h->mg[m].dev, coarse_dev, nullptr, nullptr, fine_dev, h->d_err, h->s));
    CK(cudaStreamSynchronize(h->s));
    return OHM_OK;
}

// Float32 single-grid steps of the mixed-precision inner solve (OHM_MIXED / OHM_MIXED_FF
// hierarchies), each through the kernel the V-cycle itself launches on that grid.
static int grid_setup32(ohm_hier *h, int m, const float *eta_dev, double dt, GridRef &G) {
    if (!h || h->batched || !h->mixed || m < 0 || m > (int)h->mg.size() || !eta_dev || !(dt > 0)) return OHM_ERR_INVALID;
    if (m == 0 && h->nlev > 1) return OHM_ERR_INVALID;
    G = base_ref<float>(h, m);
    CK(cudaMemcpyAsync(G.eta, eta_dev, (size_t)G.g->n() * B3 * sizeof(float), cudaMemcpyDeviceToDevice, h->s));
    CK(launch_invdiag<float>(gdev(h, *G.g), (const float *)G.eta, nullptr, h->d.lambda * dt, (float *)G.inv, h->s));
    h->eta_set = false;
    h->inv_dt = NAN;
    return OHM_OK;
}

int ohm_op_grid_sweep_f32(ohm_hier *h, int m, const float *e_in_dev, float *e_out_dev, const float *r_dev,
                          const float *eta_dev, double dt, int variant) {
    if (!e_out_dev || !r_dev || (variant != 0 && variant != 1)) return OHM_ERR_INVALID;
    GridRef G;
    int st;
    if ((st = grid_setup32(h, m, eta_dev, dt, G))) return st;
    const size_t bytes = (size_t)G.g->n() * 3 * B3 * sizeof(float);
    CK(cudaMemcpyAsync(G.r, r_dev, bytes, cudaMemcpyDeviceToDevice, h->s));
    if (e_in_dev) CK(cudaMemcpyAsync(G.e, e_in_dev, bytes, cudaMemcpyDeviceToDevice, h->s));
    const int keep = h->smoother;
    h->smoother = variant;
    st = sweeps<float>(h, G, 1, h->d.lambda * dt, e_in_dev == nullptr);
    h->smoother = keep;
    if (st) return st;
    CK(cudaMemcpyAsync(e_out_dev, G.e, bytes, cudaMemcpyDeviceToDevice, h->s));
    CK(cudaStreamSynchronize(h->s));
    return OHM_OK;
}

int ohm_op_grid_resid_restrict_f32(ohm_hier *h, int m, const float *e_dev, const float *r_dev, const float *eta_dev,
                                   double dt, float *t_dev, float *coarse_dev) {
    if (!e_dev || !r_dev || (!t_dev && !coarse_dev)) return OHM_ERR_INVALID;
    GridRef G;
    int st;
    if ((st = grid_setup32(h, m, eta_dev, dt, G))) return st;
    const bool next_blocked = m < (int)h->mg.size();
    CK(resid_restrict_base<float>(h, *G.g, e_dev, r_dev, (const float *)G.eta, h->d.lambda * dt, t_dev,
                                  next_blocked ? coarse_dev : nullptr, next_blocked ? nullptr : coarse_dev,
                                  h->small[0].data()));
    CK(cudaStreamSynchronize(h->s));
    return OHM_OK;
}

int ohm_op_grid_prolong_add_f32(ohm_hier *h, int m, const float *coarse_dev, float *fine_dev) {
    if (!h || h->batched || !h->mixed || !fine_dev || !coarse_dev) return OHM_ERR_INVALID;
    if (m < 0 || m > (int)h->mg.size() || (m == 0 && h->nlev > 1)) return OHM_ERR_INVALID;
    const HGrid &g = m == 0 ? h->amr[0] : h->mg[m - 1];
    CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->s));
    if (m == (int)h->mg.size())
        CK(launch_prolong_add<float>(gdev(h, g), nullptr, nullptr, coarse_dev, h->small[0].data(), fine_dev, h->d_err, h->s));
    else if (g.octet)
        CK(launch_prolong_add8<float>(gdev(h, h->mg[m]), coarse_dev, fine_dev, h->s));
    else
        CK(launch_prolong_add<float>(gdev(h, g), &h->mg[m].dev, coarse_dev, nullptr, nullptr, fine_dev, h->d_err, h->s));
    CK(cudaStreamSynchronize(h->s));
    return OHM_OK;
}

int ohm_op_coarsest_f32(ohm_hier *h, const float *r_dev, const float *eta_dev, double dt, float *e_dev) {
    if (!h || h->batched || !h->mixed || !r_dev || !eta_dev || !e_dev || !(dt > 0) || h->small.empty())
        return OHM_ERR_INVALID;
    const auto &d0 = h->small[0];
    const size_t n0 = (size_t)d0[0] * d0[1] * d0[2];
    const double lamdt = h->d.lambda * dt;
    CK(cudaMemcpyAsync(h->smallbuf[0].r, r_dev, 3 * n0 * sizeof(float), cudaMemcpyDeviceToDevice, h->s));
    CK(cudaMemcpyAsync(h->smallbuf[0].eta, eta_dev, n0 * sizeof(float), cudaMemcpyDeviceToDevice, h->s));
    SmallDev<float> sm = small_dev<float>(h);
    CK(launch_small_setup<float>(sm, 0.0, true, h->s));     // eta of the coarser grids
    CK(launch_small_setup<float>(sm, lamdt, false, h->s));  // inverse diagonals (paths that read them)
    h->eta_set = false;
    h->inv_dt = NAN;
    const ohm_hier_desc &d = h->d;
    const bool csb = d.nu_coarse_pre || d.nu_coarse_post;
    int st;
    if ((st = small_vcycle<float>(h, lamdt, csb ? d.nu_coarse_pre : d.nu_pre, csb ? d.nu_coarse_post : d.nu_post,
                                  d.n_coarse)))
        return st;
    CK(cudaMemcpyAsync(e_dev, h->smallbuf[0].e, 3 * n0 * sizeof(float), cudaMemcpyDeviceToDevice, h->s));
    CK(cudaStreamSynchronize(h->s));
    return OHM_OK;
}

int ohm_op_apply_L_f32(ohm_hier *h, const float *X_dev, double dt, float *out_dev) {
    if (!h || h->batched || !h->mixed || !X_dev || !out_dev || !(dt > 0) || !h->eta_set) return OHM_ERR_INVALID;
    const size_t bytes = (size_t)h->nblocks * 3 * B3 * sizeof(float);
    float *x = (float *)h->eacc;  // private copy: its covered cells are overwritten by their children's mean
    CK(cudaMemcpyAsync(x, X_dev, bytes, cudaMemcpyDeviceToDevice, h->s));
    CK(cudaMemsetAsync(out_dev, 0, bytes, h->s));  // covered blocks are not written by the operator
    int st;
    if ((st = apply_L32(h, x, nullptr, 1.0, h->d.lambda * dt, 0.0, out_dev, h->d.lambda * dt))) return st;
    CK(cudaStreamSynchronize(h->s));
    return OHM_OK;
}

}  // extern "C"
