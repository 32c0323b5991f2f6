// Host analysis of grids and partitions: integer bookkeeping that depends only
// on the grid topology and the coarse partition, never on permeability values.
//
//  * analyse_grid     -- active-cell numbering, two-point connection list
//                        (Sec. 3: one connection per interface, plus non-neighbour
//                        connections), ELL pattern of A, connection -> slot maps,
//                        and the wavefront levels of natural-order ILU(0).
//  * analyse_supports -- basis supports S_j (Sec. 5, requirement 2:
//                        Omega_j within S_j, compact), by the Cartesian box rule,
//                        the hop-distance rule for general partitions, or the
//                        block itself for constant bases.
//  * slot_layout      -- cell-major slot lists of P (block ids ascending).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <limits>
#include <numeric>
#include <string>

#include "ms_internal.h"

namespace msgb {

// Segments for the ILU(0) sweeps of any grid: maximal runs of consecutive rows
// i-1, i coupled both ways, at most max_len rows, in which no row has any
// other coupling to a row of the same run.  A sweep solves the chain of a
// segment by a scan; every other coupling leaves the segment and becomes a
// dependency on the segment holding that row.  Per direction the segments are
// handed out by wavefront level of that dependency graph (forward: couplings
// to lower rows, in ascending segment order within a level; backward:
// couplings to higher rows, descending order), so a segment's dependencies
// are always handed out before it.  Row i's neighbours (self excluded) are
// nb[deg[i] .. deg[i] + rowlen[i]), ascending.
void segment_plan(int n, const std::vector<int> &nb, const std::vector<int> &deg, const std::vector<int> &rowlen,
                  int max_len, SegmentPlan &sp) {
    auto has = [&](int i, int k) {
        auto b0 = nb.begin() + deg[i], b1 = b0 + rowlen[i];
        return std::binary_search(b0, b1, k);
    };
    std::vector<int> &off = sp.off;
    off.assign(1, 0);
    std::vector<int> stamp(n, -1);   // rows reached from the current segment by an upper coupling (k >= r + 2)
    int start = 0;
    auto mark = [&](int i) {
        for (int w = 0; w < rowlen[i]; ++w) {
            const int k = nb[deg[i] + w];
            if (k >= i + 2) stamp[k] = start;
        }
    };
    mark(0);
    for (int i = 1; i < n; ++i) {
        bool join = i - start < max_len && has(i, i - 1) && has(i - 1, i) && stamp[i] != start;
        for (int w = 0; join && w < rowlen[i]; ++w) {
            const int k = nb[deg[i] + w];
            if (k >= start && k < i - 1) join = false;
        }
        if (!join) {
            off.push_back(i);
            start = i;
        }
        mark(i);
    }
    off.push_back(n);
    const int ns = (int)off.size() - 1;
    std::vector<int> &sid = sp.sid;
    sid.assign(n, 0);
    for (int S = 0; S < ns; ++S)
        for (int i = off[S]; i < off[S + 1]; ++i) sid[i] = S;

    // couplings leaving each row's segment, and wavefront levels of the segment
    // graph: forward over couplings to lower segments (ascending order),
    // backward over couplings to higher segments (descending order)
    std::vector<int> lf(ns, 0), lb(ns, 0);
    std::vector<std::vector<int>> up(ns);
    int kgf = 0, kgb = 0;
    for (int S = 0; S < ns; ++S) {
        for (int i = off[S]; i < off[S + 1]; ++i) {
            int cf = 0, cb = 0;
            for (int w = 0; w < rowlen[i]; ++w) {
                const int k = nb[deg[i] + w];
                if (k < off[S]) { lf[S] = std::max(lf[S], lf[sid[k]] + 1); ++cf; }
                else if (k >= off[S + 1]) { up[S].push_back(sid[k]); ++cb; }
            }
            kgf = std::max(kgf, cf);
            kgb = std::max(kgb, cb);
        }
    }
    sp.kg[0] = kgf;
    sp.kg[1] = kgb;
    sp.fits = kgf <= kSegMaxKG && kgb <= kSegMaxKG;
    for (int S = ns - 1; S >= 0; --S)
        for (int d : up[S]) lb[S] = std::max(lb[S], lb[d] + 1);
    std::vector<int> &ord = sp.ord;
    ord.assign(2 * (size_t)ns, 0);
    std::iota(ord.begin(), ord.begin() + ns, 0);
    std::stable_sort(ord.begin(), ord.begin() + ns, [&](int a, int b) { return lf[a] < lf[b]; });
    for (int S = 0; S < ns; ++S) ord[(size_t)ns + S] = ns - 1 - S;
    std::stable_sort(ord.begin() + ns, ord.end(), [&](int a, int b) { return lb[a] < lb[b]; });
    sp.width = 0;
    for (const std::vector<int> *lv : {&lf, &lb}) {
        std::vector<int> cnt(ns + 1, 0);
        for (int v : *lv) sp.width = std::max(sp.width, ++cnt[v]);
    }
}

namespace {

struct Conn {
    int a, b;        // active indices, a < b not required
    int ga, gb;      // grid indices
    int8_t axis;
    double mult;
};

inline int64_t gidx(int nx, int ny, int i, int j, int k) { return i + (int64_t)nx * (j + (int64_t)ny * k); }

void plan_segments(ms_system &s, const std::vector<int> &nb, const std::vector<int> &deg,
                   const std::vector<int> &rowlen) {
    SegmentPlan sp;
    segment_plan(s.n, nb, deg, rowlen, kSegMax, sp);
    s.seg_kg[0] = sp.kg[0];
    s.seg_kg[1] = sp.kg[1];
    if (!sp.fits) {   // too many couplings per row leave a segment: not planned
        s.n_seg = 0;
        return;
    }
    s.n_seg = (int)sp.off.size() - 1;
    s.seg_width = sp.width;
    cudaStream_t st = nullptr;
    s.seg_off.upload(sp.off, st);
    s.seg_id.upload(sp.sid, st);
    s.seg_ord.upload(sp.ord, st);
    s.seg_tag.alloc(2 * (size_t)s.n);
    s.seg_tag.zero(st);   // tag 0 never matches a sweep (the sweep counter starts at 1)
}

}  // namespace

void analyse_grid(ms_system &s, const ms_grid &g) {
    MS_REQUIRE(g.nx > 0 && g.ny > 0 && g.nz > 0, MS_ERR_INVALID_ARG, "grid dimensions must be positive");
    MS_REQUIRE(g.dx > 0 && g.dy > 0 && g.dz > 0 && std::isfinite(g.dx) && std::isfinite(g.dy) && std::isfinite(g.dz),
               MS_ERR_INVALID_ARG, "cell sizes must be positive and finite");
    const int64_t N64 = (int64_t)g.nx * g.ny * g.nz;
    MS_REQUIRE(N64 < (int64_t)1 << 30, MS_ERR_INVALID_ARG, "grid too large (more than 2^30 cells)");
    const int N = (int)N64;
    s.nx = g.nx; s.ny = g.ny; s.nz = g.nz;
    s.dx = g.dx; s.dy = g.dy; s.dz = g.dz;

    s.g2a.assign(N, -1);
    s.cells.clear();
    for (int c = 0; c < N; ++c)
        if (!g.active || g.active[c]) {
            s.g2a[c] = (int)s.cells.size();
            s.cells.push_back(c);
        }
    s.n = (int)s.cells.size();
    MS_REQUIRE(s.n > 0, MS_ERR_INVALID_ARG, "grid has no active cells");

    // two-point connections in grid order: x, y, z interfaces of each cell, then NNCs
    std::vector<Conn> conns;
    conns.reserve((size_t)3 * s.n);
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int c = (int)gidx(nx, ny, i, j, k);
                int a = s.g2a[c];
                if (a < 0) continue;
                if (i + 1 < nx) {
                    double m = g.mult_x ? g.mult_x[i + (int64_t)(nx - 1) * (j + (int64_t)ny * k)] : 1.0;
                    int b = s.g2a[c + 1];
                    if (b >= 0 && m > 0) conns.push_back({a, b, c, c + 1, 0, m});
                }
                if (j + 1 < ny) {
                    double m = g.mult_y ? g.mult_y[i + (int64_t)nx * (j + (int64_t)(ny - 1) * k)] : 1.0;
                    int b = s.g2a[c + nx];
                    if (b >= 0 && m > 0) conns.push_back({a, b, c, c + nx, 1, m});
                }
                if (k + 1 < nz) {
                    double m = g.mult_z ? g.mult_z[c] : 1.0;
                    int b = s.g2a[c + nx * ny];
                    if (b >= 0 && m > 0) conns.push_back({a, b, c, c + nx * ny, 2, m});
                }
            }
    MS_REQUIRE(g.n_nnc >= 0, MS_ERR_INVALID_ARG, "n_nnc must be >= 0");
    MS_REQUIRE(g.n_nnc == 0 || (g.nnc && g.nnc_axis && g.nnc_mult), MS_ERR_INVALID_ARG, "NNC arrays missing");
    for (int e = 0; e < g.n_nnc; ++e) {
        int ca = g.nnc[2 * e], cb = g.nnc[2 * e + 1];
        int ax = g.nnc_axis[e];
        MS_REQUIRE(ca >= 0 && ca < N && cb >= 0 && cb < N && ca != cb && ax >= 0 && ax <= 2, MS_ERR_INVALID_ARG,
                   "invalid non-neighbour connection " + std::to_string(e));
        double m = g.nnc_mult[e];
        int a = s.g2a[ca], b = s.g2a[cb];
        if (a >= 0 && b >= 0 && m > 0) conns.push_back({a, b, ca, cb, (int8_t)ax, m});
    }
    s.nf = (int)conns.size();

    // neighbour lists per row -> ELL slots (ascending column, duplicates merged)
    std::vector<int> deg(s.n + 1, 0);
    for (const Conn &c : conns) { deg[c.a + 1]++; deg[c.b + 1]++; }
    for (int i = 0; i < s.n; ++i) deg[i + 1] += deg[i];
    std::vector<int> nb(deg[s.n]);
    {
        std::vector<int> fill(deg.begin(), deg.end() - 1);
        for (const Conn &c : conns) { nb[fill[c.a]++] = c.b; nb[fill[c.b]++] = c.a; }
    }
    std::vector<int> rowlen(s.n);
    int W = 0;
    for (int i = 0; i < s.n; ++i) {
        auto b0 = nb.begin() + deg[i], b1 = nb.begin() + deg[i + 1];
        std::sort(b0, b1);
        rowlen[i] = (int)(std::unique(b0, b1) - b0);
        W = std::max(W, rowlen[i]);
    }
    MS_REQUIRE(W <= 250, MS_ERR_INVALID_ARG, "a cell has more than 250 connections");
    s.W = W;
    s.h_col.assign((size_t)W * s.n, 0);
    for (int i = 0; i < s.n; ++i)
        for (int w = 0; w < W; ++w) s.h_col[(size_t)w * s.n + i] = (w < rowlen[i]) ? nb[deg[i] + w] : i;

    auto slot_of = [&](int row, int colv) -> int {
        auto b0 = nb.begin() + deg[row], b1 = b0 + rowlen[row];
        auto it = std::lower_bound(b0, b1, colv);
        return (int)(it - b0);
    };
    // row -> incident connections with the slot each one lands in
    std::vector<int> rf_ptr(s.n + 1, 0), rf_face(2 * (size_t)s.nf);
    std::vector<uint8_t> rf_slot(2 * (size_t)s.nf);
    for (const Conn &c : conns) { rf_ptr[c.a + 1]++; rf_ptr[c.b + 1]++; }
    s.rf_max = 0;
    for (int i = 0; i < s.n; ++i) s.rf_max = std::max(s.rf_max, rf_ptr[i + 1]);   // counts, before the scan
    for (int i = 0; i < s.n; ++i) rf_ptr[i + 1] += rf_ptr[i];
    {
        std::vector<int> fill(rf_ptr.begin(), rf_ptr.end() - 1);
        for (int f = 0; f < s.nf; ++f) {
            const Conn &c = conns[f];
            int p = fill[c.a]++;
            rf_face[p] = f;
            rf_slot[p] = (uint8_t)slot_of(c.a, c.b);
            p = fill[c.b]++;
            rf_face[p] = f;
            rf_slot[p] = (uint8_t)slot_of(c.b, c.a);
        }
    }

    // wavefront levels of the lower-triangular dependency graph (natural order)
    std::vector<int> lev(s.n, 0);
    int nlev = 0;
    for (int i = 0; i < s.n; ++i) {
        int l = 0;
        for (int w = 0; w < rowlen[i]; ++w) {
            int k = nb[deg[i] + w];
            if (k < i) l = std::max(l, lev[k] + 1);
        }
        lev[i] = l;
        nlev = std::max(nlev, l + 1);
    }
    std::vector<int> cnt(nlev, 0);
    for (int i = 0; i < s.n; ++i) cnt[lev[i]]++;
    std::vector<int64_t> off(nlev + 1, 0);
    for (int l = 0; l < nlev; ++l) off[l + 1] = off[l] + ((cnt[l] + 31) / 32) * 32;
    MS_REQUIRE(off[nlev] < (int64_t)1 << 31, MS_ERR_INVALID_ARG, "level layout too large");
    s.n_levels = nlev;
    s.ntot = (int)off[nlev];
    s.nnz_lower = 0;
    for (int i = 0; i < s.n; ++i)
        for (int w = 0; w < rowlen[i]; ++w) s.nnz_lower += nb[deg[i] + w] < i;
    std::vector<int> lperm(s.ntot, -1);
    {
        std::vector<int64_t> fill(off.begin(), off.end() - 1);
        for (int i = 0; i < s.n; ++i) lperm[fill[lev[i]]++] = i;
    }

    // structured grids: every cell active and every connection a Cartesian face
    s.structured = (s.n == N) && (int)(conns.size()) > 0;
    for (const Conn &c : conns)
        if (!((c.gb - c.ga == 1 && c.axis == 0) || (c.gb - c.ga == nx && c.axis == 1) ||
              (c.gb - c.ga == nx * ny && c.axis == 2))) { s.structured = false; break; }
    std::vector<int8_t> dslot;
    if (s.structured) {
        dslot.assign((size_t)6 * s.n, (int8_t)-1);
        for (const Conn &c : conns) {
            dslot[(size_t)(3 + c.axis) * s.n + c.a] = (int8_t)slot_of(c.a, c.b);   // +axis neighbour of a
            dslot[(size_t)c.axis * s.n + c.b] = (int8_t)slot_of(c.b, c.a);         // -axis neighbour of b
        }
        // CTA tile of x-pencils: TJ x TK pencils (j, k); tiles visited in
        // order of increasing J + K (a topological order of the tile DAG)
        int tk = std::min(nz, 8), tj;
        if (nz == 1) tj = std::min(512, ((ny + 31) / 32) * 32);
        else tj = std::min(256 / tk, ((ny + 31) / 32) * 32);
        if (const char *e = std::getenv("MSGB_ILU_TILE")) {     // tuning override "TJxTK"
            int a = 0, b = 0;
            if (std::sscanf(e, "%dx%d", &a, &b) == 2 && a > 0 && b > 0 && a * b <= 512) { tj = a; tk = b; }
        }
        s.TJ = tj; s.TK = tk;
        s.NJ = (ny + tj - 1) / tj; s.NK = (nz + tk - 1) / tk;
        std::vector<int> order;
        for (int d = 0; d <= s.NJ + s.NK - 2; ++d)
            for (int J = 0; J < s.NJ; ++J) {
                const int K = d - J;
                if (K >= 0 && K < s.NK) order.push_back(J + s.NJ * K);
            }
        s.tile_order.upload(order, nullptr);
        // two tagged words per value (FP64); zero tags never match a sweep
        s.face_j.alloc(std::max<size_t>((size_t)order.size() * tk * nx * 2, 1));
        s.face_k.alloc(std::max<size_t>((size_t)order.size() * tj * nx * 2, 1));
        s.face_j.zero(nullptr);
        s.face_k.zero(nullptr);
        s.tile_progress.alloc(2 * order.size());   // 16 bytes per tile (fetched with 16-byte async copies)
        s.tile_progress.zero(nullptr);
        // line-scan tiles: LTK warps (one k-row of x-lines each) x LTJ lines in j.
        // Shared memory per warp (worst case FP64 backward sweep, 4-slot ring):
        // exchange 2 + ring 4 x 5 lines of 8 bytes, plus the k-face ring.
        const int LW = 32 * (nx <= 64 ? 2 : nx <= 128 ? 4 : 8);
        if (nx <= 256) {
            const size_t per_warp = (size_t)LW * 8 * 2 + (size_t)4 * 5 * (nx + 8) * 8;
            int ltk = (int)std::min<size_t>(8, (200 * 1024 - (size_t)4 * (nx + 2) * 16) / per_warp);
            ltk = std::max(1, std::min(ltk, nz));
            int ltj = std::min(ny, 32);
            if (const char *e = std::getenv("MSGB_LINE_TILE")) {     // tuning override "TJxTK"
                int a = 0, b = 0;
                if (std::sscanf(e, "%dx%d", &a, &b) == 2 && a > 0 && b > 0 && b <= 8 &&
                    (size_t)b * per_warp + (size_t)4 * (nx + 2) * 16 <= 220 * 1024) { ltj = a; ltk = b; }
            }
            s.LTJ = ltj; s.LTK = ltk;
            s.LNJ = (ny + ltj - 1) / ltj; s.LNK = (nz + ltk - 1) / ltk;
            std::vector<int> lorder;
            for (int d = 0; d <= s.LNJ + s.LNK - 2; ++d)
                for (int J = 0; J < s.LNJ; ++J) {
                    const int K = d - J;
                    if (K >= 0 && K < s.LNK) lorder.push_back(J + s.LNJ * K);
                }
            s.line_order.upload(lorder, nullptr);
            s.lface_j.alloc((size_t)lorder.size() * ltk * nx * 2);
            s.lface_k.alloc((size_t)lorder.size() * ltj * nx * 2);
            s.line_progress.alloc(2 * lorder.size());
            s.lface_j.zero(nullptr);
            s.lface_k.zero(nullptr);
            s.line_progress.zero(nullptr);
        }
        // sweep kernels: line scan across one cluster where it can be launched,
        // else line scan over CTA tiles where the x-lines fit a warp, else pencil
        // tiles; MSGB_ILU_KERNEL=cluster|lines|pencil|generic overrides (tuning)
        plan_ilu_cluster(s);
        for (int p = 0; p < 2; ++p) {
            const int tiles = s.LTK > 0 ? 2 : 1;
            int k = s.cl_ok[p] ? 3 : tiles;
            if (const char *e = std::getenv("MSGB_ILU_KERNEL")) {
                const std::string v(e);
                if (v == "cluster") k = s.cl_ok[p] ? 3 : tiles;
                else if (v == "lines") k = tiles;
                else if (v == "pencil") k = 1;
                else if (v == "generic") k = 0;
                else if (v == "level") k = 4;
            }
            s.ilu_kind[p] = k;
        }
    } else {
        // any grid: segment dataflow sweeps; MSGB_ILU_KERNEL=level selects the
        // level-synchronous sweeps (one cooperative launch), =generic the
        // flag-ordered sweeps
        plan_segments(s, nb, deg, rowlen);
        const char *e = std::getenv("MSGB_ILU_KERNEL");
        const std::string v = e ? std::string(e) : std::string();
        const int k = v == "generic" ? 0 : v == "level" ? 4 : (s.n_seg > 0 ? 5 : 4);
        s.ilu_kind[0] = s.ilu_kind[1] = k;
    }

    // host copies + device upload
    s.h_fa.resize(s.nf);
    s.h_fb.resize(s.nf);
    std::vector<int> ga(s.nf), gb(s.nf);
    std::vector<int8_t> ax(s.nf);
    std::vector<double> mu(s.nf);
    for (int f = 0; f < s.nf; ++f) {
        s.h_fa[f] = conns[f].a; s.h_fb[f] = conns[f].b;
        ga[f] = conns[f].ga; gb[f] = conns[f].gb;
        ax[f] = conns[f].axis; mu[f] = conns[f].mult;
    }
    cudaStream_t st = nullptr;
    s.f_a.upload(s.h_fa, st);
    s.f_b.upload(s.h_fb, st);
    s.f_ga.upload(ga, st);
    s.f_gb.upload(gb, st);
    s.f_axis.upload(ax, st);
    s.f_mult.upload(mu, st);
    s.f_T.alloc(std::max(s.nf, 1));
    s.rf_ptr.upload(rf_ptr, st);
    s.rf_face.upload(rf_face, st);
    s.rf_slot.upload(rf_slot, st);
    s.col.upload(s.h_col, st);
    if (s.structured) s.dir_slot.upload(dslot, st);
    s.lperm.upload(lperm, st);
    {
        std::vector<int> lo(off.size());
        for (size_t l = 0; l < off.size(); ++l) lo[l] = (int)off[l];
        s.lev_off.upload(lo, st);
        s.lev_bar.alloc(2);
        s.lev_bar.zero(st);
    }
    size_t en = std::max<size_t>((size_t)W * s.n, 1);
    s.off_u.alloc(en); s.off_p.alloc(en); s.diag.alloc(s.n);
    s.flags.alloc(s.n);
    s.flags.zero(st);
    s.sync.alloc(kSyncWords);
    s.sync.zero(st);
    MS_CUDA(cudaStreamSynchronize(st));
}

// Cartesian block of every active cell; empty blocks dropped, the rest
// numbered in Cartesian block order.
int partition_cartesian(const ms_system &s, int bx, int by, int bz, std::vector<int> &part) {
    MS_REQUIRE(bx > 0 && by > 0 && bz > 0, MS_ERR_INVALID_ARG, "block sizes must be positive");
    const int64_t nbx = (s.nx + bx - 1) / bx, nby = (s.ny + by - 1) / by, nbz = (s.nz + bz - 1) / bz;
    MS_REQUIRE(nbx * nby * nbz < ((int64_t)1 << 31), MS_ERR_INVALID_ARG, "too many Cartesian blocks");
    std::vector<int> id(nbx * nby * nbz, -1);
    part.resize(s.n);
    for (int a = 0; a < s.n; ++a) {
        const int c = s.cells[a];
        const int64_t I = (c % s.nx) / bx, J = ((c / s.nx) % s.ny) / by, K = (c / (s.nx * s.ny)) / bz;
        part[a] = (int)(I + nbx * (J + nby * K));
        id[part[a]] = 0;
    }
    int M = 0;
    for (auto &v : id)
        if (v == 0) v = M++;
    for (int a = 0; a < s.n; ++a) part[a] = id[part[a]];
    return M;
}

// ------------------------------------------------------------------ supports
namespace {

// Cells of each block (ascending active index).
void block_members(const std::vector<int> &part, int M, std::vector<int> &bptr, std::vector<int> &bcell) {
    bptr.assign(M + 1, 0);
    for (int b : part) bptr[b + 1]++;
    for (int j = 0; j < M; ++j) bptr[j + 1] += bptr[j];
    bcell.resize(part.size());
    std::vector<int> fill(bptr.begin(), bptr.end() - 1);
    for (int i = 0; i < (int)part.size(); ++i) bcell[fill[part[i]]++] = i;
}

}  // namespace

void analyse_supports(const ms_system &s, const std::vector<int> &part, int M, int rule, int bx, int by, int bz,
                      std::vector<int> &cptr, std::vector<int> &ccell) {
    const int n = s.n, W = s.W;
    std::vector<int> bptr, bcell;
    block_members(part, M, bptr, bcell);
    for (int j = 0; j < M; ++j)
        MS_REQUIRE(bptr[j + 1] > bptr[j], MS_ERR_INVALID_ARG, "partition block " + std::to_string(j) + " is empty");
    auto nbr = [&](int i, int w) { return s.h_col[(size_t)w * n + i]; };
    cptr.assign(M + 1, 0);
    ccell.clear();

    if (rule == MS_SUPPORT_BLOCK) {
        for (int j = 0; j < M; ++j) {
            ccell.insert(ccell.end(), bcell.begin() + bptr[j], bcell.begin() + bptr[j + 1]);
            cptr[j + 1] = (int)ccell.size();
        }
        return;
    }

    if (rule == MS_SUPPORT_BOX) {
        MS_REQUIRE(bx > 0 && by > 0 && bz > 0, MS_ERR_INVALID_ARG, "box support needs a positive block size");
        // mark[c] == 2j+1: inside block j's grown box; 2j+2: reached
        std::vector<int> mark(n, 0);
        std::vector<int> frontier;
        for (int j = 0; j < M; ++j) {
            const int c0 = s.cells[bcell[bptr[j]]];
            const int x = c0 % s.nx, y = (c0 / s.nx) % s.ny, z = c0 / (s.nx * s.ny);
            const int I = x / bx, J = y / by, K = z / bz;
            const int lo[3] = {std::max(0, I * bx - bx / 2), std::max(0, J * by - by / 2),
                               std::max(0, K * bz - bz / 2)};
            const int hi[3] = {std::min(s.nx - 1, (I + 1) * bx - 1 + bx / 2),
                               std::min(s.ny - 1, (J + 1) * by - 1 + by / 2),
                               std::min(s.nz - 1, (K + 1) * bz - 1 + bz / 2)};
            const int in = 2 * j + 1, seen = 2 * j + 2;
            for (int zz = lo[2]; zz <= hi[2]; ++zz)
                for (int yy = lo[1]; yy <= hi[1]; ++yy)
                    for (int xx = lo[0]; xx <= hi[0]; ++xx) {
                        int a = s.g2a[gidx(s.nx, s.ny, xx, yy, zz)];
                        if (a >= 0) mark[a] = in;
                    }
            frontier.assign(bcell.begin() + bptr[j], bcell.begin() + bptr[j + 1]);
            for (int a : frontier) mark[a] = seen;
            size_t start = ccell.size();
            for (size_t h = 0; h < frontier.size(); ++h) {
                int a = frontier[h];
                ccell.push_back(a);
                for (int w = 0; w < W; ++w) {
                    int k = nbr(a, w);
                    if (mark[k] == in) { mark[k] = seen; frontier.push_back(k); }
                }
            }
            std::sort(ccell.begin() + start, ccell.end());
            cptr[j + 1] = (int)ccell.size();
        }
        return;
    }

    MS_REQUIRE(rule == MS_SUPPORT_HOP, MS_ERR_INVALID_ARG, "unknown support rule");
    // centre cell of each block: nearest to the index-space centroid, lowest index on ties
    std::vector<int> centre(M);
    for (int j = 0; j < M; ++j) {
        double cx = 0, cy = 0, cz = 0;
        const int m = bptr[j + 1] - bptr[j];
        for (int p = bptr[j]; p < bptr[j + 1]; ++p) {
            int c = s.cells[bcell[p]];
            cx += c % s.nx; cy += (c / s.nx) % s.ny; cz += c / (s.nx * s.ny);
        }
        cx /= m; cy /= m; cz /= m;
        double best = std::numeric_limits<double>::infinity();
        for (int p = bptr[j]; p < bptr[j + 1]; ++p) {
            int c = s.cells[bcell[p]];
            double ex = c % s.nx - cx, ey = (c / s.nx) % s.ny - cy, ez = c / (s.nx * s.ny) - cz;
            double d2 = ex * ex + ey * ey + ez * ez;
            if (d2 < best) { best = d2; centre[j] = bcell[p]; }
        }
    }
    std::vector<int> dist_blk(n, -1), dist_ctr(n, -1);
    std::vector<int> seen_blk(M, -1);
    std::vector<int> q1, q2, cand;
    for (int j = 0; j < M; ++j) {
        cand.assign(bcell.begin() + bptr[j], bcell.begin() + bptr[j + 1]);
        std::vector<int> adj;
        for (int p = bptr[j]; p < bptr[j + 1]; ++p)
            for (int w = 0; w < W; ++w) {
                int k = part[nbr(bcell[p], w)];
                if (k != j && seen_blk[k] != j) { seen_blk[k] = j; adj.push_back(k); }
            }
        for (int k : adj) {
            auto inside = [&](int c) { int b = part[c]; return b == j || b == k; };
            q1.assign(bcell.begin() + bptr[j], bcell.begin() + bptr[j + 1]);
            for (int a : q1) dist_blk[a] = 0;
            for (size_t h = 0; h < q1.size(); ++h) {
                int a = q1[h];
                for (int w = 0; w < W; ++w) {
                    int c = nbr(a, w);
                    if (inside(c) && dist_blk[c] < 0) { dist_blk[c] = dist_blk[a] + 1; q1.push_back(c); }
                }
            }
            q2.assign(1, centre[k]);
            dist_ctr[centre[k]] = 0;
            for (size_t h = 0; h < q2.size(); ++h) {
                int a = q2[h];
                for (int w = 0; w < W; ++w) {
                    int c = nbr(a, w);
                    if (inside(c) && dist_ctr[c] < 0) { dist_ctr[c] = dist_ctr[a] + 1; q2.push_back(c); }
                }
            }
            for (int p = bptr[k]; p < bptr[k + 1]; ++p) {
                int a = bcell[p];
                if (dist_blk[a] >= 0 && (dist_ctr[a] < 0 || dist_blk[a] <= dist_ctr[a])) cand.push_back(a);
            }
            for (int a : q1) dist_blk[a] = -1;
            for (int a : q2) dist_ctr[a] = -1;
        }
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        ccell.insert(ccell.end(), cand.begin(), cand.end());
        cptr[j + 1] = (int)ccell.size();
    }
}

void slot_layout(const ms_system &s, const std::vector<int> &part, int M, const std::vector<int> &cptr,
                 const std::vector<int> &ccell, int &B, std::vector<int> &pid, std::vector<int> &csrc,
                 std::vector<unsigned char> &is_home) {
    const int n = s.n;
    std::vector<int> cnt(n, 0);
    for (int c : ccell) cnt[c]++;
    B = 0;
    for (int i = 0; i < n; ++i) {
        MS_REQUIRE(cnt[i] > 0, MS_ERR_INVALID_ARG, "a cell is covered by no basis support");
        B = std::max(B, cnt[i]);
    }
    pid.assign((size_t)B * n, kSlotPad);
    is_home.assign((size_t)B * n, 0);
    csrc.resize(ccell.size());
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int j = 0; j < M; ++j)             // increasing j -> ascending ids per cell
        for (int e = cptr[j]; e < cptr[j + 1]; ++e) {
            int i = ccell[e];
            int sl = cnt[i]++;
            size_t at = (size_t)sl * n + i;
            pid[at] = j;
            is_home[at] = (part[i] == j);
            csrc[e] = (int)at;
        }
}

}  // namespace msgb
