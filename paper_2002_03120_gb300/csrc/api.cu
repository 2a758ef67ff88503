// api.cu -- the C ABI of libsdpd (include/sdpd.h): context life cycle,
// parameter validation, per-instance grids, the stage sequence of
// Algorithm 1 and its CUDA-graph replay.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

using namespace sdpd;

namespace {

thread_local std::string g_last_error = "";

sdpd_status fail(sdpd_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}

#define CUDA_TRY(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail(SDPD_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
    } while (0)

struct HostInst {
    sdpd_params P;
    long long n = 0, begin = 0;
    bool set = false;
    double xmin[3] = { 0, 0, 0 }, xmax[3] = { 0, 0, 0 };
    double Rmax = 0.0;
    std::vector<int> type;
};

}  // namespace

void sdpd::set_last_error(const char *msg) { g_last_error = msg; }

struct sdpd_ctx {
    int n_inst = 0, precision = 0, cap = 384, K = 16;
    long long N = 0, Npad = 0;
    std::vector<HostInst> hi;
    std::vector<Inst> inst;
    Bufs b{};
    std::vector<void *> allocs;        // fixed-size buffers
    std::vector<void *> geo_allocs;    // buffers sized by the grid / rigid count
    Inst *d_inst = nullptr;
    int any_filter = 0, any_artvis = 0, any_reinit = 0;
    std::vector<double> probe_y;   // mean slab positions of the last viscosity probe
    int newton3 = 1;                   // force pass: 1 half-pair (Newton 3), 0 direct, 2/3 pair stream,
                                       // 4 half-pair with pushed results (FP32), 5 direct with
                                       // fewer registers (FP32)
    int noise_cache = 1;               // second evaluation of a step reuses the first one's normals
    double skin = 0.03;                // Verlet skin as a fraction of h
    int cell_sub = 1;                  // cells per minimum cell width: 1 (27-cell stencil) or 2 (125)
    bool geometry_ready = false, cells_valid = false, density_valid = false, drag_valid = false;
    int sticky_err = 0;
    long long host_step = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    cudaGraph_t graph_def = nullptr;
};

namespace {

template <class T> sdpd_status dalloc(sdpd_ctx *c, T **p, size_t count, bool geo = false)
{
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(SDPD_E_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    (geo ? c->geo_allocs : c->allocs).push_back((void *)*p);
    return SDPD_OK;
}

#define ALLOC(ptr, n, geo)                                                                      \
    do {                                                                                        \
        sdpd_status s_ = dalloc(c, &(ptr), (size_t)(n), geo);                                   \
        if (s_ != SDPD_OK) return s_;                                                           \
    } while (0)

void free_geo(sdpd_ctx *c)
{
    for (void *p : c->geo_allocs) cudaFree(p);
    c->geo_allocs.clear();
}

void drop_graph(sdpd_ctx *c)
{
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->graph_def) cudaGraphDestroy(c->graph_def);
    c->graph = nullptr;
    c->graph_def = nullptr;
}

double lucy_W(double r, double h)
{
    if (r >= h) return 0.0;
    const double q = r / h, om = 1.0 - q;
    return 105.0 / (16.0 * PI * h * h * h) * (1.0 + 3.0 * q) * om * om * om;
}

// Normalisation of the kernel coefficient: C_n = 1 / (dx^3 * sum of W over a
// perfect cubic lattice, self included).
double kernel_norm(double dx, double h)
{
    const int m = (int)std::ceil(h / dx) + 1;
    double s = 0.0;
    for (int k = -m; k <= m; ++k)
        for (int j = -m; j <= m; ++j)
            for (int i = -m; i <= m; ++i) s += lucy_W(std::sqrt((double)(i * i + j * j + k * k)) * dx, h);
    return 1.0 / (dx * dx * dx * s);
}

sdpd_status validate(const sdpd_params &p, int k)
{
    char buf[256];
    auto bad = [&](const char *what) {
        std::snprintf(buf, sizeof buf, "instance %d: %s", k, what);
        return fail(SDPD_E_INVALID, buf);
    };
    if (!(p.dx > 0) || !(p.r_c > 0) || !(p.dt > 0) || !(p.rho0 > 0)) return bad("dx, r_c, dt, rho0 must be > 0");
    if (!(p.eta >= 0) || !(p.kBT >= 0)) return bad("eta and kBT must be >= 0");
    const double Ca = 20.0 * p.eta / 3.0 - 4.0 * p.xi, Cb = 17.0 * p.xi - 40.0 * p.eta / 3.0;
    const double tol = 1e-12 * (p.eta > 0 ? p.eta : 1.0);
    if (Ca < -tol || Cb < -tol) return bad("need 40 eta/51 <= xi <= 5 eta/3 (gamma^a, gamma^b >= 0)");
    for (int a = 0; a < 3; ++a) {
        if (!(p.box[a] > 0)) return bad("box must be > 0");
        if (p.periodic[a] && p.box[a] < 3.0 * p.r_c) return bad("periodic axis narrower than 3 r_c");
    }
    if (p.body_axis < 0 || p.body_axis > 2 || p.split_axis < 0 || p.split_axis > 2) return bad("axis out of range");
    if (p.dem_law == 1 && !(p.restitution > 0 && p.restitution <= 1)) return bad("restitution must be in (0, 1]");
    if (p.dem_law == 0 && !(p.E_p > 0)) return bad("E_p must be > 0 for dem_law 0");
    if (p.mu_fric < 0) return bad("mu_fric must be >= 0");
    return SDPD_OK;
}

uint32_t morton(int x, int y, int z)
{
    return morton_spread((uint32_t)x) | (morton_spread((uint32_t)y) << 1) | (morton_spread((uint32_t)z) << 2);
}

// Grids, Morton ranks, rigid lists and the per-instance constants; sized
// buffers are (re)allocated here.
sdpd_status prepare(sdpd_ctx *c)
{
    for (int k = 0; k < c->n_inst; ++k)
        if (!c->hi[k].set) return fail(SDPD_E_STATE, "sdpd_set_particles not called for every instance");
    drop_graph(c);
    free_geo(c);
    c->inst.assign(c->n_inst, Inst{});
    std::vector<int> rank_all;
    int cell_base = 0;
    for (int k = 0; k < c->n_inst; ++k) {
        const HostInst &H = c->hi[k];
        const sdpd_params &p = H.P;
        Inst &I = c->inst[k];
        std::memset(&I, 0, sizeof(I));
        // the skin shrinks where a periodic axis could not hold 3 cells with it
        double skin = c->skin;
        for (int a = 0; a < 3; ++a)
            if (p.periodic[a]) {
                const double room = (p.box[a] / 3.0 - std::max(p.r_c, 2.0 * H.Rmax)) / p.r_c;
                skin = std::min(skin, std::max(0.0, room * 0.999));
            }
        const double rb = p.r_c * (1.0 + skin);
        // cmin bounds the reach of any listed pair; cells are cmin / sub wide
        // and the stencil reaches sub cells each way
        const double cmin = std::max(rb, 2.0 * H.Rmax + skin * p.r_c);
        const int sub = c->cell_sub;
        const double cw = cmin / sub;
        I.sub = sub;
        for (int a = 0; a < 3; ++a) {
            I.origin[a] = p.origin[a];
            I.box[a] = p.box[a];
            I.periodic[a] = p.periodic[a] ? 1 : 0;
            if (p.periodic[a]) {
                // 3 cells of cmin fit, so at least 2 sub + 1 cells of cw do:
                // the stencil never meets the same cell twice
                int nc = (int)std::floor(p.box[a] / cw);
                if (nc < 3 || (int)std::floor(p.box[a] / cmin) < 3) {
                    char buf[160];
                    std::snprintf(buf, sizeof buf,
                                  "instance %d axis %d: periodic box must hold 3 cells of max(h, 2 R_max)", k, a);
                    return fail(SDPD_E_INVALID, buf);
                }
                I.nc[a] = nc;
                I.cs[a] = p.box[a] / nc;
                I.lo[a] = p.origin[a];
            } else {
                const double lo = std::min(H.xmin[a], p.origin[a]) - 0.5 * cmin;
                const double hi = std::max(H.xmax[a], p.origin[a] + p.box[a]) + 0.5 * cmin;
                I.cs[a] = cw;
                I.lo[a] = lo;
                I.nc[a] = (int)std::ceil((hi - lo) / cw);
            }
            if (I.nc[a] > 1023) return fail(SDPD_E_INVALID, "more than 1023 cells on an axis");
            I.inv_cs[a] = 1.0 / I.cs[a];
            I.csf[a] = (float)I.cs[a];
        }
        I.ncell = I.nc[0] * I.nc[1] * I.nc[2];
        I.cell_base = cell_base;
        // Morton rank of each linear cell
        std::vector<std::pair<uint32_t, int>> codes(I.ncell);
        for (int z = 0; z < I.nc[2]; ++z)
            for (int y = 0; y < I.nc[1]; ++y)
                for (int x = 0; x < I.nc[0]; ++x) {
                    const int lin = (z * I.nc[1] + y) * I.nc[0] + x;
                    codes[lin] = { morton(x, y, z), lin };
                }
        std::sort(codes.begin(), codes.end());
        std::vector<int> rank(I.ncell);
        for (int r = 0; r < I.ncell; ++r) rank[codes[r].second] = r;
        rank_all.insert(rank_all.end(), rank.begin(), rank.end());
        cell_base += I.ncell;
        I.p_begin = H.begin;
        I.p_end = H.begin + H.n;
        // physics constants
        const double h = p.r_c;
        I.dx = p.dx; I.rc = h; I.rc2 = h * h; I.inv_rc = 1.0 / h; I.dt = p.dt; I.hdt = 0.5 * p.dt;
        I.isqrt_dt = 1.0 / std::sqrt(p.dt);
        I.Wc = 105.0 / (16.0 * PI * h * h * h);
        I.Fc = 315.0 / (4.0 * PI * h * h * h * h * h);
        I.W0 = I.Wc;
        I.Cn = kernel_norm(p.dx, h);
        I.mf = p.rho0 * p.dx * p.dx * p.dx;
        I.inv_dx3 = 1.0 / (p.dx * p.dx * p.dx);
        I.rho0 = p.rho0; I.p0 = p.p0; I.alpha = p.alpha; I.beta_p = p.beta_p;
        I.alpha_int = (p.alpha >= 1.0 && p.alpha <= 32.0 && p.alpha == std::floor(p.alpha)) ? (int)p.alpha : 0;
        I.eta = p.eta; I.kBT = p.kBT;
        I.Ca = std::max(0.0, 20.0 * p.eta / 3.0 - 4.0 * p.xi);
        I.Cb = std::max(0.0, 17.0 * p.xi - 40.0 * p.eta / 3.0);
        I.Ka = 2.0 * std::sqrt(p.kBT * I.Ca * I.Fc);
        I.Kb = 2.0 * std::sqrt(p.kBT * I.Cb * I.Fc);
        I.coeff_c = p.coeff_c; I.coeff_d = p.coeff_d; I.coeff_r = p.coeff_r; I.coeff_t = p.coeff_t;
        for (int a = 0; a < 3; ++a) I.g[a] = p.g[a];
        I.body_amp = p.body_amp; I.body_axis = p.body_axis; I.split_axis = p.split_axis;
        I.filter = p.pressure_filter ? 1 : 0; I.clamp = p.clamp_negative_p ? 1 : 0;
        I.reinit = p.density_reinit ? 1 : 0;
        I.artvis = p.artvis ? 1 : 0; I.dem_law = p.dem_law;
        I.noise = (p.coeff_t != 0.0 && p.kBT > 0.0) ? 1 : 0;
        I.artvis_rlim = p.artvis_alpha * p.dx; I.artvis_e = p.artvis_e;
        I.kn = p.kn; I.kt_ratio = 1.0 / (2.0 * (1.0 + p.nu_p));
        if (p.dem_law == 1) {
            const double le = std::log(p.restitution);
            I.zeta = -le / std::sqrt(PI * PI + le * le);
        }
        I.nu_p = p.nu_p; I.E_p = p.E_p; I.mu_fric = p.mu_fric;
        I.lub_gap_min = p.lub_gap_min; I.eps_min = p.eps_min;
        I.Vf = 4.0 / 3.0 * PI * h * h * h;
        I.lever_fluid = 0.5 * p.dx;
        I.key0 = (uint32_t)(p.seed & 0xFFFFFFFFull);
        I.key1 = (uint32_t)(p.seed >> 32) ^ (uint32_t)k;
        I.rcf = (float)h; I.inv_rcf = (float)(1.0 / h);
        I.Wcf = (float)I.Wc; I.Fcf = (float)I.Fc; I.W0f = (float)I.W0;
        I.Caf = (float)I.Ca; I.Cbf = (float)I.Cb; I.Kaf = (float)I.Ka; I.Kbf = (float)I.Kb;
        I.isqrt_dtf = (float)I.isqrt_dt;
        I.coeff_cf = (float)p.coeff_c; I.coeff_df = (float)p.coeff_d;
        I.coeff_rf = (float)p.coeff_r; I.coeff_tf = (float)p.coeff_t;
        I.lever_fluidf = (float)I.lever_fluid;
        I.rb = rb;
        I.rb2 = rb * rb;
        I.half_skin = 0.5 * skin * h;
        for (int a = 0; a < 3; ++a) {
            I.dom_hi[a] = I.origin[a] + I.box[a];
            const double hb = 0.5 * I.box[a];
            std::memcpy(&I.hbox_bits[a], &hb, sizeof hb);
        }
        I.rb2f = (float)(rb * rb * (1.0 + 1e-5));
        I.guard_lo = (float)(I.rc2 * (1.0 - 1e-5));
        I.guard_hi = (float)(I.rc2 * (1.0 + 1e-5));
        I.artvis_r2f_hi = (float)(I.artvis_rlim * I.artvis_rlim * (1.0 + 1e-5));
    }
    Bufs &b = c->b;
    b.ncell_total = cell_base;
    b.cell_sub = c->cell_sub;
    int *rank_d = nullptr;
    ALLOC(rank_d, cell_base, true);
    CUDA_TRY(cudaMemcpy(rank_d, rank_all.data(), sizeof(int) * cell_base, cudaMemcpyHostToDevice));
    b.cell_rank = rank_d;
    // neighbour cells of every cell (offsets -sub..sub per axis), ascending
    // key, with the offset code (ox+2) + 5 (oy+2) + 25 (oz+2): neighbour
    // lists then come out sorted by slot.  Cells are split over host threads.
    {
        if (cell_base >= (1 << 24)) return fail(SDPD_E_INVALID, "too many cells");
        std::vector<int> adj((size_t)cell_base * ADJ, -1);
        std::vector<int> inst_of(cell_base);
        for (int k = 0; k < c->n_inst; ++k)
            std::fill(inst_of.begin() + c->inst[k].cell_base,
                      inst_of.begin() + c->inst[k].cell_base + c->inst[k].ncell, k);
        auto fill = [&](int lin0, int lin1) {
            std::pair<int, int> nbs[ADJ];
            for (int gl = lin0; gl < lin1; ++gl) {
                const Inst &I = c->inst[inst_of[gl]];
                const int lin = gl - I.cell_base, d = I.sub;
                const int x = lin % I.nc[0], y = (lin / I.nc[0]) % I.nc[1], z = lin / (I.nc[0] * I.nc[1]);
                const int key = I.cell_base + rank_all[gl];
                int nn = 0;
                for (int oz = -d; oz <= d; ++oz)
                    for (int oy = -d; oy <= d; ++oy)
                        for (int ox = -d; ox <= d; ++ox) {
                            int cc[3] = { x + ox, y + oy, z + oz };
                            bool ok = true;
                            for (int a = 0; a < 3; ++a) {
                                if (I.periodic[a]) cc[a] = (cc[a] + I.nc[a]) % I.nc[a];
                                else if (cc[a] < 0 || cc[a] >= I.nc[a]) ok = false;
                            }
                            if (!ok) continue;
                            const int l2 = (cc[2] * I.nc[1] + cc[1]) * I.nc[0] + cc[0];
                            const int k2 = I.cell_base + rank_all[I.cell_base + l2];
                            nbs[nn++] = { k2, (ox + 2) + 5 * (oy + 2) + 25 * (oz + 2) };
                        }
                std::sort(nbs, nbs + nn);
                for (int q = 0; q < nn; ++q) adj[(size_t)key * ADJ + q] = (nbs[q].first << 7) | nbs[q].second;
            }
        };
        const int nth = std::max(1, std::min((int)std::thread::hardware_concurrency(),
                                             std::min(16, cell_base / 4096 + 1)));
        if (nth == 1) {
            fill(0, cell_base);
        } else {
            std::vector<std::thread> pool;
            for (int t = 0; t < nth; ++t)
                pool.emplace_back(fill, (int)((long long)cell_base * t / nth),
                                  (int)((long long)cell_base * (t + 1) / nth));
            for (auto &th : pool) th.join();
        }
        int *adj_d = nullptr;
        ALLOC(adj_d, adj.size(), true);
        CUDA_TRY(cudaMemcpy(adj_d, adj.data(), sizeof(int) * adj.size(), cudaMemcpyHostToDevice));
        b.cell_adj = adj_d;
    }
    ALLOC(b.ccount, cell_base, true);
    ALLOC(b.cstart, cell_base + 1, true);
    ALLOC(b.scan_partials, (cell_base + 1023) / 1024 + 1, true);
    // rigid lists (gid order)
    std::vector<int> rigid_gid, rigid_of(c->N, -1);
    for (int k = 0; k < c->n_inst; ++k) {
        const HostInst &H = c->hi[k];
        for (long long i = 0; i < H.n; ++i)
            if (H.type[i] == T_RIGID) {
                rigid_of[H.begin + i] = (int)rigid_gid.size();
                rigid_gid.push_back((int)(H.begin + i));
            }
    }
    b.nrigid = (int)rigid_gid.size();
    ALLOC(b.rigid_gid, b.nrigid, true);
    ALLOC(b.rigid_of, c->N, true);
    if (b.nrigid) CUDA_TRY(cudaMemcpy(b.rigid_gid, rigid_gid.data(), sizeof(int) * b.nrigid, cudaMemcpyHostToDevice));
    if (c->N) CUDA_TRY(cudaMemcpy(b.rigid_of, rigid_of.data(), sizeof(int) * c->N, cudaMemcpyHostToDevice));
    const size_t nr1 = b.nrigid ? (size_t)b.nrigid : 1;
    ALLOC(b.eps, nr1, true);
    ALLOC(b.fdg, 3 * nr1, true);
    ALLOC(b.dsum, 5 * nr1, true);
    const size_t nk = nr1 * c->K;
    ALLOC(b.h_n, nr1, true);
    ALLOC(b.hn_n, nr1, true);
    ALLOC(b.h_part, nk, true);
    ALLOC(b.hn_part, nk, true);
    ALLOC(b.h_del, 3 * nk, true);
    ALLOC(b.hn_del, 3 * nk, true);
    CUDA_TRY(cudaMemset(b.h_n, 0, sizeof(int) * nr1));
    CUDA_TRY(cudaMemset(b.hn_n, 0, sizeof(int) * nr1));
    CUDA_TRY(cudaMemset(b.eps, 0, sizeof(double) * nr1));
    CUDA_TRY(cudaMemset(b.fdg, 0, sizeof(double) * 3 * nr1));
    if (!c->d_inst) {
        sdpd_status s = dalloc(c, &c->d_inst, c->n_inst, false);
        if (s != SDPD_OK) return s;
    }
    CUDA_TRY(cudaMemcpy(c->d_inst, c->inst.data(), sizeof(Inst) * c->n_inst, cudaMemcpyHostToDevice));
    b.inst = c->d_inst;
    c->any_filter = 0;
    c->any_reinit = 0;
    c->any_artvis = 0;
    for (auto &I : c->inst) {
        c->any_filter |= I.filter;
        c->any_reinit |= I.reinit;
        c->any_artvis |= I.artvis;
    }
    c->geometry_ready = true;
    c->cells_valid = c->density_valid = c->drag_valid = false;
    return SDPD_OK;
}

sdpd_status check_err(sdpd_ctx *c)
{
    int e = 0;
    CUDA_TRY(cudaMemcpy(&e, c->b.err, sizeof(int), cudaMemcpyDeviceToHost));
    c->sticky_err |= e;
    e = c->sticky_err;
    if (!e) return SDPD_OK;
    if (e & ERR_NBR_CAP) return fail(SDPD_E_CAPACITY, "neighbour list capacity exceeded (raise max_neighbors)");
    if (e & ERR_CONTACT_CAP) return fail(SDPD_E_CAPACITY, "contact history capacity exceeded (raise max_contacts)");
    if (e & ERR_CELL_CAP) return fail(SDPD_E_CAPACITY, "cell capacity exceeded");
    if (e & ERR_PAIR_CAP) return fail(SDPD_E_CAPACITY, "pair buffer capacity exceeded");
    if (e & ERR_REV) return fail(SDPD_E_STATE, "neighbour lists not symmetric");
    if (e & ERR_NONFINITE) return fail(SDPD_E_NONFINITE, "non-finite position, velocity or spin");
    if (e & ERR_DOMAIN) return fail(SDPD_E_DOMAIN, "particle outside the grid (crossed a wall axis, or moved more than a box length in one step)");
    return fail(SDPD_E_CUDA, "unknown device error");
}

sdpd_status ensure_geometry(sdpd_ctx *c)
{
    if (!c->geometry_ready) return prepare(c);
    return SDPD_OK;
}

// force modes with the Newton-3 half-pair pass (1: pull gather in FP32,
// 4: push); they need the reverse index of the lists
inline bool half_pairs(int mode) { return mode == 1 || mode == 4; }

void enqueue_build(sdpd_ctx *c, cudaStream_t st, const int *gate = nullptr)
{
    c->b.use_cache = c->noise_cache;
    launch_build(c->b, c->precision, half_pairs(c->newton3), gate, st);
}

}  // namespace

// ======================================================================= ABI
extern "C" {

const char *sdpd_last_error(void) { return g_last_error.c_str(); }

sdpd_status sdpd_init(const sdpd_params *params, int n_instances, const long long *n_particles,
                      int precision, int max_neighbors, int max_contacts, sdpd_ctx **out)
{
    if (!out) return fail(SDPD_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!params || !n_particles || n_instances < 1) return fail(SDPD_E_INVALID, "bad instance list");
    if (precision != SDPD_PREC_FP64 && precision != SDPD_PREC_SPLIT) return fail(SDPD_E_INVALID, "bad precision");
    if (max_neighbors < 0 || max_neighbors > SDPD_MAX_NEIGHBORS)
        return fail(SDPD_E_INVALID, "max_neighbors must be in [0, SDPD_MAX_NEIGHBORS]");
    if (max_contacts < 0) return fail(SDPD_E_INVALID, "negative max_contacts");
    for (int k = 0; k < n_instances; ++k) {
        if (n_particles[k] < 0) return fail(SDPD_E_INVALID, "negative particle count");
        sdpd_status s = validate(params[k], k);
        if (s != SDPD_OK) return s;
    }
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0)
        return fail(SDPD_E_CUDA, "no CUDA device");
    init_pair_kernels();   // kernel attributes, set outside any stream capture
    init_cell_kernels();
    sdpd_ctx *c = new sdpd_ctx();
    c->n_inst = n_instances;
    c->precision = precision;
    c->cap = max_neighbors > 0 ? max_neighbors : 384;
    c->K = max_contacts > 0 ? max_contacts : 16;
    c->hi.resize(n_instances);
    long long N = 0;
    for (int k = 0; k < n_instances; ++k) {
        c->hi[k].P = params[k];
        c->hi[k].n = n_particles[k];
        c->hi[k].begin = N;
        N += n_particles[k];
    }
    if (N >= (1LL << 31) - 1) {
        delete c;
        return fail(SDPD_E_INVALID, "more than 2^31 particles");
    }
    c->N = N;
    c->Npad = (N + 127) / 128 * 128;
    Bufs &b = c->b;
    b.N = N;
    b.Npad = c->Npad;
    b.n_inst = n_instances;
    b.cap = c->cap;
    b.K = c->K;
    b.pair_block = 128;
    b.tpp = 1;
    b.cell_sub = 1;
    auto cleanup = [&](sdpd_status s) {
        sdpd_destroy(c);
        return s;
    };
#define IALLOC(ptr, n)                                                                          \
    do {                                                                                        \
        sdpd_status s_ = dalloc(c, &(ptr), (size_t)(n), false);                                 \
        if (s_ != SDPD_OK) return cleanup(s_);                                                  \
    } while (0)
    const size_t n3 = 3 * (size_t)N;
    IALLOC(b.x, n3); IALLOC(b.v, n3); IALLOC(b.w, n3); IALLOC(b.F, n3); IALLOC(b.T, n3);
    IALLOC(b.dv, n3);
    IALLOC(b.type, N); IALLOC(b.pinst, N);
    IALLOC(b.R, N); IALLOC(b.m, N); IALLOC(b.Iner, N); IALLOC(b.rm, N); IALLOC(b.rI, N);
    IALLOC(b.key, N); IALLOC(b.slot_in_cell, N); IALLOC(b.tmp_perm, N); IALLOC(b.perm, N);
    IALLOC(b.slot_of, N); IALLOC(b.stype, N);
    IALLOC(b.sd, N); IALLOC(b.sp, N); IALLOC(b.sp2, N);
    IALLOC(b.rxn, N); IALLOC(b.rxn32, N);
    IALLOC(b.A32, N);
    if (precision == SDPD_PREC_SPLIT) {
        IALLOC(b.B32, N); IALLOC(b.C32, N); IALLOC(b.D32, N);
    } else {
        IALLOC(b.A64, N); IALLOC(b.B64, N); IALLOC(b.C64, N); IALLOC(b.D64, N);
    }
    IALLOC(b.nbr, (size_t)c->cap * c->Npad);
    IALLOC(b.ncnt, N);
    IALLOC(b.nfirst, N);
    IALLOC(b.skey, N);
    IALLOC(b.nbflag, N);
    IALLOC(b.rev, (size_t)c->cap * c->Npad);
    // each particle owns about half of its list (hash ownership, spread of a
    // few pairs): the pair buffer and the normals cache of the Newton-3 pass
    // hold cap/2 + 64 rows.  The direct pass instead caches the normals of
    // every list entry ([cap][Npad]).  A context runs one force pass at a
    // time, so both layouts share one arena.
    b.capown = std::min(c->cap, c->cap / 2 + 64);
    {
        const size_t rs = (precision == SDPD_PREC_SPLIT) ? sizeof(float) : sizeof(double);
        const size_t Np = (size_t)c->Npad, own = (size_t)b.capown * Np, all = (size_t)c->cap * Np;
        // {f, h.x} / {o, ce} in resA; {h.y, h.z} in resB (pushed results)
        const size_t n_resA = 4 * rs * own, n_resB = 2 * rs * own;
        const size_t n_zA = 4 * rs * own, n_zB = 2 * rs * own;
        const size_t half_bytes = n_resA + n_resB + n_zA + n_zB, direct_bytes = 6 * rs * all;
        char *arena = nullptr, *oa = nullptr, *ob = nullptr, *dummy = nullptr;
        IALLOC(arena, std::max(half_bytes, direct_bytes));
        IALLOC(dummy, 16);
        IALLOC(oa, 4 * rs * (size_t)N);
        IALLOC(ob, 2 * rs * (size_t)N);
        b.resA = arena;
        b.resB = n_resB ? arena + n_resA : dummy;
        b.zA = arena + n_resA + n_resB;
        b.zB = arena + n_resA + n_resB + n_zA;
        b.zdA = arena;
        b.zdB = arena + 4 * rs * all;
        b.ownA = oa; b.ownB = ob;
    }
    IALLOC(b.xl64, N); IALLOC(b.dsp, N);
    IALLOC(b.aclose, N); IALLOC(b.aclose_ok, 1); IALLOC(b.sdr, N); IALLOC(b.xs, 3 * N);
    IALLOC(b.need_build, 1); IALLOC(b.fresh, 1);
    IALLOC(b.list_epoch, 1); IALLOC(b.cache_epoch, 1); IALLOC(b.cache_step, 1);
    b.use_cache = 1;
    IALLOC(b.step, 1); IALLOC(b.err, 1); IALLOC(b.pair_count, 1); IALLOC(b.work, 1);
    IALLOC(b.probe, 4096 * 3 + 64);
#undef IALLOC
    if (cudaMemset(b.rev, 0, sizeof(uint16_t) * (size_t)c->cap * c->Npad) != cudaSuccess ||
        cudaMemset(b.need_build, 0, sizeof(int)) != cudaSuccess || cudaMemset(b.fresh, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(b.aclose_ok, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(b.list_epoch, 0, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(b.cache_epoch, 0xFF, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(b.cache_step, 0xFF, sizeof(long long)) != cudaSuccess)
        return cleanup(fail(SDPD_E_CUDA, "cudaMemset failed"));
    if (cudaMemset(b.err, 0, sizeof(int)) != cudaSuccess || cudaMemset(b.step, 0, sizeof(long long)) != cudaSuccess ||
        cudaMemset(b.F, 0, sizeof(double) * (n3 ? n3 : 1)) != cudaSuccess ||
        cudaMemset(b.T, 0, sizeof(double) * (n3 ? n3 : 1)) != cudaSuccess)
        return cleanup(fail(SDPD_E_CUDA, "cudaMemset failed"));
    // per-instance pinst
    std::vector<int> pinst(N);
    for (int k = 0; k < n_instances; ++k)
        for (long long i = 0; i < n_particles[k]; ++i) pinst[c->hi[k].begin + i] = k;
    if (N && cudaMemcpy(b.pinst, pinst.data(), sizeof(int) * N, cudaMemcpyHostToDevice) != cudaSuccess)
        return cleanup(fail(SDPD_E_CUDA, "cudaMemcpy pinst"));
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return cleanup(fail(SDPD_E_CUDA, "cudaStreamCreate"));
    *out = c;
    return SDPD_OK;
}

void sdpd_destroy(sdpd_ctx *c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    drop_graph(c);
    free_geo(c);
    for (void *p : c->allocs) cudaFree(p);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

sdpd_status sdpd_set_particles(sdpd_ctx *c, int inst, long long n, const double *x, const double *v,
                               const double *w, const int *type, const double *radius, const double *mass)
{
    if (!c || inst < 0 || inst >= c->n_inst) return fail(SDPD_E_INVALID, "bad context or instance");
    HostInst &H = c->hi[inst];
    if (n != H.n) return fail(SDPD_E_INVALID, "particle count differs from sdpd_init");
    if (n && (!x || !v || !w || !type || !radius || !mass)) return fail(SDPD_E_INVALID, "NULL array");
    const size_t n3 = 3 * (size_t)n;
    std::vector<double> hx(n3), hv(n3), hw(n3), hR(n), hm(n), hI(n);
    std::vector<int> ht(n);
    if (n) {
        CUDA_TRY(cudaMemcpy(hx.data(), x, sizeof(double) * n3, cudaMemcpyDefault));
        CUDA_TRY(cudaMemcpy(hv.data(), v, sizeof(double) * n3, cudaMemcpyDefault));
        CUDA_TRY(cudaMemcpy(hw.data(), w, sizeof(double) * n3, cudaMemcpyDefault));
        CUDA_TRY(cudaMemcpy(ht.data(), type, sizeof(int) * n, cudaMemcpyDefault));
        CUDA_TRY(cudaMemcpy(hR.data(), radius, sizeof(double) * n, cudaMemcpyDefault));
        CUDA_TRY(cudaMemcpy(hm.data(), mass, sizeof(double) * n, cudaMemcpyDefault));
    }
    const sdpd_params &p = H.P;
    double Rmax = 0.0;
    for (int a = 0; a < 3; ++a) {
        H.xmin[a] = 1e300;
        H.xmax[a] = -1e300;
    }
    for (long long i = 0; i < n; ++i) {
        const int t = ht[i];
        if (t < 0 || t > 3) return fail(SDPD_E_INVALID, "particle type must be 0..3");
        if (!(hm[i] > 0.0)) return fail(SDPD_E_INVALID, "particle mass must be > 0");
        for (int a = 0; a < 3; ++a) {
            const double xa = hx[3 * i + a];
            if (!std::isfinite(xa)) return fail(SDPD_E_NONFINITE, "non-finite input position");
            if (p.periodic[a] && (xa < p.origin[a] || xa >= p.origin[a] + p.box[a]))
                return fail(SDPD_E_DOMAIN, "position outside the periodic box");
            H.xmin[a] = std::min(H.xmin[a], xa);
            H.xmax[a] = std::max(H.xmax[a], xa);
        }
        if (t == T_RIGID) {
            if (!(hR[i] > 0.0)) return fail(SDPD_E_INVALID, "rigid radius must be > 0");
            Rmax = std::max(Rmax, hR[i]);
        }
        // moment of inertia of a solid sphere, 2/5 m a^2, a = R (rigid) or
        // dx/2 (fluid): the --iner input of Table 1 has no printed value
        const double arm = (t == T_RIGID) ? hR[i] : 0.5 * p.dx;
        hI[i] = 0.4 * hm[i] * arm * arm;
    }
    if (Rmax != H.Rmax || !H.set) c->geometry_ready = false;
    H.Rmax = Rmax;
    H.type = ht;
    H.set = true;
    Bufs &b = c->b;
    const long long o = H.begin;
    if (n) {
        CUDA_TRY(cudaMemcpy(b.x + 3 * o, hx.data(), sizeof(double) * n3, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(b.v + 3 * o, hv.data(), sizeof(double) * n3, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(b.w + 3 * o, hw.data(), sizeof(double) * n3, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(b.type + o, ht.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(b.R + o, hR.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(b.m + o, hm.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(b.Iner + o, hI.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
        // correctly rounded reciprocals (IEEE division on the host) for the
        // update's divisions by m and I
        std::vector<double> hrm(n), hrI(n);
        for (long long i = 0; i < n; ++i) {
            hrm[i] = hm[i] != 0.0 ? 1.0 / hm[i] : 0.0;
            hrI[i] = hI[i] != 0.0 ? 1.0 / hI[i] : 0.0;
        }
        CUDA_TRY(cudaMemcpy(b.rm + o, hrm.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(b.rI + o, hrI.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemset(b.F + 3 * o, 0, sizeof(double) * n3));
        CUDA_TRY(cudaMemset(b.T + 3 * o, 0, sizeof(double) * n3));
    }
    // the grid depends on the extents on wall axes: always re-derive it
    c->geometry_ready = false;
    c->cells_valid = c->density_valid = c->drag_valid = false;
    c->sticky_err = 0;
    CUDA_TRY(cudaMemset(b.err, 0, sizeof(int)));
    return SDPD_OK;
}

sdpd_status sdpd_upload_state(sdpd_ctx *c, const double *x, const double *v, const double *w, void *stream)
{
    if (!c) return fail(SDPD_E_INVALID, "NULL context");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * 3 * (size_t)c->N;
    (void)cudaGetLastError();
    if (c->cells_valid) {
        // keep the lists: move the particles by their displacement and let
        // the gated build of the next step decide (half the skin)
        if (x) CUDA_TRY(cudaMemcpyAsync(c->b.xs, x, bytes, cudaMemcpyDefault, st));
        if (v) CUDA_TRY(cudaMemcpyAsync(c->b.v, v, bytes, cudaMemcpyDefault, st));
        if (w) CUDA_TRY(cudaMemcpyAsync(c->b.w, w, bytes, cudaMemcpyDefault, st));
        launch_absorb(c->b, c->precision, c->b.xs, x ? 1 : 0, st);
        CUDA_TRY(cudaGetLastError());
        if (x) c->density_valid = false;
        c->drag_valid = false;
        return SDPD_OK;
    }
    if (x) CUDA_TRY(cudaMemcpyAsync(c->b.x, x, bytes, cudaMemcpyDefault, st));
    if (v) CUDA_TRY(cudaMemcpyAsync(c->b.v, v, bytes, cudaMemcpyDefault, st));
    if (w) CUDA_TRY(cudaMemcpyAsync(c->b.w, w, bytes, cudaMemcpyDefault, st));
    c->cells_valid = c->density_valid = c->drag_valid = false;
    return SDPD_OK;
}

sdpd_status sdpd_download_state(sdpd_ctx *c, double *x, double *v, double *w, double *F, double *N, void *stream)
{
    if (!c) return fail(SDPD_E_INVALID, "NULL context");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * 3 * (size_t)c->N;
    if (x) CUDA_TRY(cudaMemcpyAsync(x, c->b.x, bytes, cudaMemcpyDefault, st));
    if (v) CUDA_TRY(cudaMemcpyAsync(v, c->b.v, bytes, cudaMemcpyDefault, st));
    if (w) CUDA_TRY(cudaMemcpyAsync(w, c->b.w, bytes, cudaMemcpyDefault, st));
    if (F) CUDA_TRY(cudaMemcpyAsync(F, c->b.F, bytes, cudaMemcpyDefault, st));
    if (N) CUDA_TRY(cudaMemcpyAsync(N, c->b.T, bytes, cudaMemcpyDefault, st));
    return SDPD_OK;
}

namespace {
// checkpoint image: header, x v w [N][3] (gid order), contact histories
struct CkptHeader {
    uint32_t magic, version;
    long long n, nrigid, K, step;
};
constexpr uint32_t CKPT_MAGIC = 0x4B434453u;  // "SDCK"
long long ckpt_bytes(const sdpd_ctx *c)
{
    const long long nr = c->b.nrigid, K = c->K;
    return (long long)sizeof(CkptHeader) + 9LL * c->N * (long long)sizeof(double) +
           (nr + nr * K) * (long long)sizeof(int) + 3LL * nr * K * (long long)sizeof(double);
}
}  // namespace

sdpd_status sdpd_checkpoint_size(sdpd_ctx *c, long long *bytes)
{
    if (!c || !bytes) return fail(SDPD_E_INVALID, "sdpd_checkpoint_size: NULL argument");
    sdpd_status s = ensure_geometry(c);   // the rigid-particle count is known from here on
    if (s != SDPD_OK) return s;
    *bytes = ckpt_bytes(c);
    return SDPD_OK;
}

sdpd_status sdpd_checkpoint(sdpd_ctx *c, void *buf, long long bytes)
{
    if (!c || !buf) return fail(SDPD_E_INVALID, "sdpd_checkpoint: NULL argument");
    sdpd_status g = ensure_geometry(c);
    if (g != SDPD_OK) return g;
    if (bytes < ckpt_bytes(c)) return fail(SDPD_E_INVALID, "sdpd_checkpoint: buffer too small");
    CUDA_TRY(cudaDeviceSynchronize());
    sdpd_status e = check_err(c);
    if (e != SDPD_OK) return e;
    char *p = (char *)buf;
    CkptHeader h{ CKPT_MAGIC, 1u, c->N, c->b.nrigid, c->K, 0 };
    CUDA_TRY(cudaMemcpy(&h.step, c->b.step, sizeof(long long), cudaMemcpyDeviceToHost));
    std::memcpy(p, &h, sizeof h);
    p += sizeof h;
    const size_t n3 = sizeof(double) * 3 * (size_t)c->N;
    CUDA_TRY(cudaMemcpy(p, c->b.x, n3, cudaMemcpyDeviceToHost)); p += n3;
    CUDA_TRY(cudaMemcpy(p, c->b.v, n3, cudaMemcpyDeviceToHost)); p += n3;
    CUDA_TRY(cudaMemcpy(p, c->b.w, n3, cudaMemcpyDeviceToHost)); p += n3;
    const size_t nr = (size_t)c->b.nrigid, nk = nr * (size_t)c->K;
    if (nr) {
        CUDA_TRY(cudaMemcpy(p, c->b.h_n, sizeof(int) * nr, cudaMemcpyDeviceToHost)); p += sizeof(int) * nr;
        CUDA_TRY(cudaMemcpy(p, c->b.h_part, sizeof(int) * nk, cudaMemcpyDeviceToHost)); p += sizeof(int) * nk;
        CUDA_TRY(cudaMemcpy(p, c->b.h_del, sizeof(double) * 3 * nk, cudaMemcpyDeviceToHost));
    }
    // the next step rebuilds the lists, as it does after a restore, so both
    // continuations sum the same terms in the same order
    c->cells_valid = c->density_valid = c->drag_valid = false;
    return SDPD_OK;
}

sdpd_status sdpd_restore(sdpd_ctx *c, const void *buf, long long bytes)
{
    if (!c || !buf) return fail(SDPD_E_INVALID, "sdpd_restore: NULL argument");
    if (bytes < (long long)sizeof(CkptHeader)) return fail(SDPD_E_INVALID, "sdpd_restore: image too small");
    const char *p = (const char *)buf;
    CkptHeader h;
    std::memcpy(&h, p, sizeof h);
    p += sizeof h;
    if (h.magic != CKPT_MAGIC || h.version != 1u) return fail(SDPD_E_INVALID, "sdpd_restore: not a checkpoint image");
    sdpd_status g = ensure_geometry(c);   // prepares a fresh context (rigid lists, histories)
    if (g != SDPD_OK) return g;
    if (h.n != c->N || h.nrigid != c->b.nrigid || h.K != c->K)
        return fail(SDPD_E_INVALID, "sdpd_restore: image of another context shape (particles, spheres, contacts)");
    if (bytes < ckpt_bytes(c)) return fail(SDPD_E_INVALID, "sdpd_restore: image truncated");
    CUDA_TRY(cudaDeviceSynchronize());
    const size_t n3 = sizeof(double) * 3 * (size_t)c->N;
    CUDA_TRY(cudaMemcpy(c->b.x, p, n3, cudaMemcpyHostToDevice)); p += n3;
    CUDA_TRY(cudaMemcpy(c->b.v, p, n3, cudaMemcpyHostToDevice)); p += n3;
    CUDA_TRY(cudaMemcpy(c->b.w, p, n3, cudaMemcpyHostToDevice)); p += n3;
    const size_t nr = (size_t)c->b.nrigid, nk = nr * (size_t)c->K;
    if (nr) {
        CUDA_TRY(cudaMemcpy(c->b.h_n, p, sizeof(int) * nr, cudaMemcpyHostToDevice)); p += sizeof(int) * nr;
        CUDA_TRY(cudaMemcpy(c->b.h_part, p, sizeof(int) * nk, cudaMemcpyHostToDevice)); p += sizeof(int) * nk;
        CUDA_TRY(cudaMemcpy(c->b.h_del, p, sizeof(double) * 3 * nk, cudaMemcpyHostToDevice));
    }
    CUDA_TRY(cudaMemcpy(c->b.step, &h.step, sizeof(long long), cudaMemcpyHostToDevice));
    c->host_step = h.step;
    c->cells_valid = c->density_valid = c->drag_valid = false;
    return SDPD_OK;
}

sdpd_status sdpd_set_step(sdpd_ctx *c, long long step)
{
    if (!c) return fail(SDPD_E_INVALID, "NULL context");
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpy(c->b.step, &step, sizeof(long long), cudaMemcpyHostToDevice));
    c->host_step = step;
    return SDPD_OK;
}

sdpd_status sdpd_get_step(sdpd_ctx *c, long long *step)
{
    if (!c || !step) return fail(SDPD_E_INVALID, "NULL argument");
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpy(step, c->b.step, sizeof(long long), cudaMemcpyDeviceToHost));
    return SDPD_OK;
}

sdpd_status sdpd_build_count(sdpd_ctx *c, long long *builds)
{
    if (!c || !builds) return fail(SDPD_E_INVALID, "NULL argument");
    CUDA_TRY(cudaDeviceSynchronize());
    unsigned e = 0;
    CUDA_TRY(cudaMemcpy(&e, c->b.list_epoch, sizeof(unsigned), cudaMemcpyDeviceToHost));
    *builds = (long long)e;
    return SDPD_OK;
}

sdpd_status sdpd_build_cells(sdpd_ctx *c, void *stream)
{
    if (!c) return fail(SDPD_E_INVALID, "NULL context");
    (void)cudaGetLastError();  // launch errors below are this call's own
    sdpd_status s = ensure_geometry(c);
    if (s != SDPD_OK) return s;
    enqueue_build(c, (cudaStream_t)stream);
    CUDA_TRY(cudaGetLastError());
    c->cells_valid = true;
    c->density_valid = c->drag_valid = false;
    return SDPD_OK;
}

sdpd_status sdpd_compute_density(sdpd_ctx *c, void *stream)
{
    if (!c) return fail(SDPD_E_INVALID, "NULL context");
    (void)cudaGetLastError();  // launch errors below are this call's own
    if (!c->cells_valid) return fail(SDPD_E_STATE, "sdpd_build_cells must precede sdpd_compute_density");
    launch_density(c->b, c->precision, c->any_filter | (c->any_reinit << 1) | (c->any_artvis << 2), half_pairs(c->newton3), nullptr, (cudaStream_t)stream);
    CUDA_TRY(cudaGetLastError());
    c->density_valid = true;
    return SDPD_OK;
}

sdpd_status sdpd_couple_drag(sdpd_ctx *c, void *stream)
{
    if (!c) return fail(SDPD_E_INVALID, "NULL context");
    (void)cudaGetLastError();  // launch errors below are this call's own
    if (!c->density_valid) return fail(SDPD_E_STATE, "sdpd_compute_density must precede sdpd_couple_drag");
    launch_drag(c->b, c->precision, (cudaStream_t)stream);
    CUDA_TRY(cudaGetLastError());
    c->drag_valid = true;
    return SDPD_OK;
}

sdpd_status sdpd_compute_forces(sdpd_ctx *c, int velver, void *stream)
{
    if (!c) return fail(SDPD_E_INVALID, "NULL context");
    (void)cudaGetLastError();  // launch errors below are this call's own
    if (velver != 1 && velver != 2) return fail(SDPD_E_INVALID, "velver must be 1 or 2");
    if (!c->drag_valid) return fail(SDPD_E_STATE, "sdpd_couple_drag must precede sdpd_compute_forces");
    launch_forces(c->b, c->precision, velver, c->newton3, (cudaStream_t)stream);
    CUDA_TRY(cudaGetLastError());
    return SDPD_OK;
}

sdpd_status sdpd_integrate(sdpd_ctx *c, int velver, void *stream)
{
    if (!c) return fail(SDPD_E_INVALID, "NULL context");
    (void)cudaGetLastError();  // launch errors below are this call's own
    if (velver != 1 && velver != 2) return fail(SDPD_E_INVALID, "velver must be 1 or 2");
    if (!c->geometry_ready || !c->b.inst) return fail(SDPD_E_STATE, "no forces computed yet");
    cudaStream_t st = (cudaStream_t)stream;
    launch_integrate(c->b, c->precision, velver, c->any_artvis, st);
    if (velver == 2) {
        launch_step_done(c->b, st);
        c->host_step += 1;
    }
    CUDA_TRY(cudaGetLastError());
    if (velver == 1) c->cells_valid = c->density_valid = false;
    c->drag_valid = false;
    return SDPD_OK;
}

sdpd_status sdpd_step(sdpd_ctx *c, long long n_steps, void *stream)
{
    if (!c) return fail(SDPD_E_INVALID, "NULL context");
    (void)cudaGetLastError();  // launch errors below are this call's own
    if (n_steps < 0) return fail(SDPD_E_INVALID, "negative step count");
    cudaStream_t st = (cudaStream_t)stream;
    sdpd_status s = ensure_geometry(c);
    if (s != SDPD_OK) return s;
    if (!c->cells_valid) {
        enqueue_build(c, st);
        c->cells_valid = true;
        c->density_valid = false;
    }
    if (!c->density_valid) {
        launch_density(c->b, c->precision, c->any_filter | (c->any_reinit << 1) | (c->any_artvis << 2), half_pairs(c->newton3), nullptr, st);
        c->density_valid = true;
    }
    if (!c->graph) {
        // one full step; positions are unchanged between the velver-2 build
        // and the next step's velver 1, so that sub-step reuses the build and
        // the density exactly
        CUDA_TRY(cudaStreamSynchronize(st));
        CUDA_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        // Verlet skin: the list is rebuilt only when a drift has used up half
        // the skin (device flag gating the build kernels); density is redone
        // at velver 1 only after such a build, at velver 2 always
        cudaStream_t cs = c->cap_stream;
        enqueue_build(c, cs, c->b.need_build);
        launch_density(c->b, c->precision, c->any_filter | (c->any_reinit << 1) | (c->any_artvis << 2), half_pairs(c->newton3), c->b.fresh, cs);
        launch_drag(c->b, c->precision, cs);
        launch_forces(c->b, c->precision, 1, c->newton3, cs);
        launch_integrate(c->b, c->precision, 1, c->any_artvis, cs);
        enqueue_build(c, cs, c->b.need_build);
        launch_density(c->b, c->precision, c->any_filter | (c->any_reinit << 1) | (c->any_artvis << 2), half_pairs(c->newton3), nullptr, cs);
        launch_drag(c->b, c->precision, cs);
        launch_forces(c->b, c->precision, 2, c->newton3, cs);
        launch_integrate(c->b, c->precision, 2, c->any_artvis, cs);
        launch_step_done(c->b, cs);
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &c->graph_def);
        if (e != cudaSuccess) return fail(SDPD_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&c->graph, c->graph_def, 0);
        if (e != cudaSuccess) return fail(SDPD_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    for (long long k = 0; k < n_steps; ++k) CUDA_TRY(cudaGraphLaunch(c->graph, st));
    c->host_step += n_steps;
    CUDA_TRY(cudaStreamSynchronize(st));
    c->cells_valid = c->density_valid = true;
    c->drag_valid = false;
    return check_err(c);
}

sdpd_status sdpd_set_force_mode(sdpd_ctx *c, int newton3)
{
    if (!c) return fail(SDPD_E_INVALID, "NULL context");
    if (newton3 < 0 || newton3 > 5) return fail(SDPD_E_INVALID, "force mode must be in 0..5");
    CUDA_TRY(cudaDeviceSynchronize());
    if (newton3 != c->newton3) {
        c->newton3 = newton3;
        drop_graph(c);
        c->cells_valid = c->density_valid = c->drag_valid = false;
    }
    return SDPD_OK;
}

sdpd_status sdpd_set_noise_cache(sdpd_ctx *c, int on)
{
    if (!c) return fail(SDPD_E_INVALID, "NULL context");
    if (on != 0 && on != 1) return fail(SDPD_E_INVALID, "on must be 0 or 1");
    CUDA_TRY(cudaDeviceSynchronize());
    if (on != c->noise_cache) {
        c->noise_cache = on;
        drop_graph(c);
        c->cells_valid = c->density_valid = c->drag_valid = false;
    }
    return SDPD_OK;
}

sdpd_status sdpd_set_block_size(sdpd_ctx *c, int threads)
{
    if (!c) return fail(SDPD_E_INVALID, "NULL context");
    if (threads != 64 && threads != 128 && threads != 256) return fail(SDPD_E_INVALID, "block size must be 64, 128 or 256");
    CUDA_TRY(cudaDeviceSynchronize());
    if (threads != c->b.pair_block) {
        c->b.pair_block = threads;
        drop_graph(c);
    }
    return SDPD_OK;
}

sdpd_status sdpd_set_threads_per_particle(sdpd_ctx *c, int tpp)
{
    if (!c) return fail(SDPD_E_INVALID, "NULL context");
    if (tpp != 1 && tpp != 2 && tpp != 4) return fail(SDPD_E_INVALID, "threads per particle must be 1, 2 or 4");
    CUDA_TRY(cudaDeviceSynchronize());
    if (tpp != c->b.tpp) {
        c->b.tpp = tpp;
        drop_graph(c);
    }
    return SDPD_OK;
}

sdpd_status sdpd_set_cell_factor(sdpd_ctx *c, int sub)
{
    if (!c) return fail(SDPD_E_INVALID, "NULL context");
    if (sub != 1 && sub != 2) return fail(SDPD_E_INVALID, "cells per minimum width must be 1 or 2");
    CUDA_TRY(cudaDeviceSynchronize());
    if (sub != c->cell_sub) {
        c->cell_sub = sub;
        c->geometry_ready = false;
        drop_graph(c);
        c->cells_valid = c->density_valid = c->drag_valid = false;
    }
    return SDPD_OK;
}

sdpd_status sdpd_set_skin(sdpd_ctx *c, double skin)
{
    if (!c) return fail(SDPD_E_INVALID, "NULL context");
    if (!(skin >= 0.0 && skin <= 0.5)) return fail(SDPD_E_INVALID, "skin must be in [0, 0.5]");
    CUDA_TRY(cudaDeviceSynchronize());
    if (skin != c->skin) {
        c->skin = skin;
        c->geometry_ready = false;
        drop_graph(c);
        c->cells_valid = c->density_valid = c->drag_valid = false;
    }
    return SDPD_OK;
}

sdpd_status sdpd_graph_kernels(sdpd_ctx *c, long long *n_kernels)
{
    if (!c || !n_kernels) return fail(SDPD_E_INVALID, "bad argument");
    *n_kernels = 0;
    if (!c->graph_def) return SDPD_OK;
    size_t n = 0;
    CUDA_TRY(cudaGraphGetNodes(c->graph_def, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    CUDA_TRY(cudaGraphGetNodes(c->graph_def, nodes.data(), &n));
    long long k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        CUDA_TRY(cudaGraphNodeGetType(nd, &t));
        k += (t == cudaGraphNodeTypeKernel);
    }
    *n_kernels = k;
    return SDPD_OK;
}

sdpd_status sdpd_check(sdpd_ctx *c)
{
    if (!c) return fail(SDPD_E_INVALID, "NULL context");
    CUDA_TRY(cudaDeviceSynchronize());
    return check_err(c);
}

sdpd_status sdpd_viscosity_probe(sdpd_ctx *c, int inst, int n_bins, double *profile_out, double *mu_app_out)
{
    if (!c || inst < 0 || inst >= c->n_inst) return fail(SDPD_E_INVALID, "bad context or instance");
    if (n_bins < 1 || n_bins > 4096) return fail(SDPD_E_INVALID, "n_bins must be in 1..4096");
    sdpd_status s = ensure_geometry(c);
    if (s != SDPD_OK) return s;
    CUDA_TRY(cudaDeviceSynchronize());
    launch_probe(c->b, inst, n_bins, 0, c->hi[inst].n);
    std::vector<double> h(3 * n_bins + 4);
    CUDA_TRY(cudaMemcpy(h.data(), c->b.probe, sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
    for (int k = 0; k < n_bins; ++k)
        if (profile_out) profile_out[k] = h[n_bins + k] > 0 ? h[k] / h[n_bins + k] : 0.0;
    // mean position of each slab's particles (for sdpd_viscosity_fit)
    c->probe_y.assign(n_bins, -1.0);
    for (int k = 0; k < n_bins; ++k)
        if (h[n_bins + k] > 0) c->probe_y[k] = h[2 * n_bins + 4 + k] / h[n_bins + k];
    const sdpd_params &p = c->hi[inst].P;
    const double V = 0.5 * (h[2 * n_bins] / std::max(h[2 * n_bins + 2], 1.0) +
                            h[2 * n_bins + 1] / std::max(h[2 * n_bins + 3], 1.0));
    const double D = 0.5 * p.box[p.split_axis];
    if (mu_app_out) *mu_app_out = p.rho0 * p.body_amp * D * D / (12.0 * V);
    return check_err(c);
}

sdpd_status sdpd_viscosity_fit(sdpd_ctx *c, int inst, int n_bins, double *mu_fit_out)
{
    if (!mu_fit_out) return fail(SDPD_E_INVALID, "sdpd_viscosity_fit: NULL output");
    std::vector<double> prof(n_bins > 0 ? n_bins : 1);
    double mu_mean = 0.0;
    sdpd_status s = sdpd_viscosity_probe(c, inst, n_bins, prof.data(), &mu_mean);
    if (s != SDPD_OK) return s;
    const sdpd_params &p = c->hi[inst].P;
    const int a = p.split_axis;
    const double L = p.box[a], h = p.r_c;
    double mu_sum = 0.0;
    for (int half = 0; half < 2; ++half) {
        // least squares v = c0 + c1 t + c2 t^2 over the slabs of this half whose
        // centres lie at least h from its ends (walls or splitting planes)
        const double y0 = half * 0.5 * L, y1 = y0 + 0.5 * L, ym = 0.5 * (y0 + y1);
        double S[5] = { 0, 0, 0, 0, 0 }, T[3] = { 0, 0, 0 };
        int used = 0;
        for (int k = 0; k < n_bins; ++k) {
            const double y = c->probe_y[k];   // mean position of the slab's particles
            if (y < 0.0 || y < y0 + h || y > y1 - h) continue;
            const double t = y - ym, v = prof[k];
            double tp = 1.0;
            for (int e = 0; e < 5; ++e) { S[e] += tp; tp *= t; }
            T[0] += v; T[1] += v * t; T[2] += v * t * t;
            ++used;
        }
        if (used < 4) return fail(SDPD_E_INVALID, "sdpd_viscosity_fit: fewer than 4 slabs h away from the ends of a half");
        // normal equations [S0 S1 S2; S1 S2 S3; S2 S3 S4] c = T, Cramer's rule for c2
        const double M[3][3] = { { S[0], S[1], S[2] }, { S[1], S[2], S[3] }, { S[2], S[3], S[4] } };
        auto det3 = [](const double m[3][3]) {
            return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
                   m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
        };
        double M2[3][3];
        for (int r = 0; r < 3; ++r) {
            M2[r][0] = M[r][0];
            M2[r][1] = M[r][1];
            M2[r][2] = T[r];
        }
        const double c2 = det3(M2) / det3(M);
        // steady state: mu v'' = -rho g on the lower half (+g), +rho g above
        const double g = half == 0 ? p.body_amp : -p.body_amp;
        mu_sum += -p.rho0 * g / (2.0 * c2);
    }
    *mu_fit_out = 0.5 * mu_sum;
    return SDPD_OK;
}

sdpd_status sdpd_get_state(sdpd_ctx *c, int inst, double *x, double *v, double *w, double *F, double *N,
                           double *d, double *p)
{
    if (!c || inst < 0 || inst >= c->n_inst) return fail(SDPD_E_INVALID, "bad context or instance");
    CUDA_TRY(cudaDeviceSynchronize());
    const HostInst &H = c->hi[inst];
    const size_t n3 = 3 * (size_t)H.n;
    const long long o = H.begin;
    if (H.n) {
        if (x) CUDA_TRY(cudaMemcpy(x, c->b.x + 3 * o, sizeof(double) * n3, cudaMemcpyDeviceToHost));
        if (v) CUDA_TRY(cudaMemcpy(v, c->b.v + 3 * o, sizeof(double) * n3, cudaMemcpyDeviceToHost));
        if (w) CUDA_TRY(cudaMemcpy(w, c->b.w + 3 * o, sizeof(double) * n3, cudaMemcpyDeviceToHost));
        if (F) CUDA_TRY(cudaMemcpy(F, c->b.F + 3 * o, sizeof(double) * n3, cudaMemcpyDeviceToHost));
        if (N) CUDA_TRY(cudaMemcpy(N, c->b.T + 3 * o, sizeof(double) * n3, cudaMemcpyDeviceToHost));
        if ((d || p) && c->density_valid) {
            std::vector<int> slot(H.n);
            std::vector<double> sd(c->N), sp(c->N);
            CUDA_TRY(cudaMemcpy(slot.data(), c->b.slot_of + o, sizeof(int) * H.n, cudaMemcpyDeviceToHost));
            CUDA_TRY(cudaMemcpy(sd.data(), c->b.sd, sizeof(double) * c->N, cudaMemcpyDeviceToHost));
            CUDA_TRY(cudaMemcpy(sp.data(), c->b.sp2, sizeof(double) * c->N, cudaMemcpyDeviceToHost));
            for (long long i = 0; i < H.n; ++i) {
                if (d) d[i] = sd[slot[i]];
                if (p) p[i] = sp[slot[i]];
            }
        } else if (d || p) {
            return fail(SDPD_E_STATE, "density not computed for the current positions");
        }
    }
    return check_err(c);
}

sdpd_status sdpd_get_drag(sdpd_ctx *c, int inst, double *eps, double *F_dg)
{
    if (!c || inst < 0 || inst >= c->n_inst) return fail(SDPD_E_INVALID, "bad context or instance");
    CUDA_TRY(cudaDeviceSynchronize());
    const HostInst &H = c->hi[inst];
    int r0 = 0, nr = 0;
    for (int k = 0; k < c->n_inst; ++k) {
        int cnt = 0;
        for (int t : c->hi[k].type) cnt += (t == T_RIGID);
        if (k < inst) r0 += cnt;
        if (k == inst) nr = cnt;
    }
    (void)H;
    if (nr) {
        if (eps) CUDA_TRY(cudaMemcpy(eps, c->b.eps + r0, sizeof(double) * nr, cudaMemcpyDeviceToHost));
        if (F_dg) CUDA_TRY(cudaMemcpy(F_dg, c->b.fdg + 3 * r0, sizeof(double) * 3 * nr, cudaMemcpyDeviceToHost));
    }
    return check_err(c);
}

sdpd_status sdpd_get_pairs(sdpd_ctx *c, int inst, long long cap, int *ij, long long *n_out)
{
    if (!c || inst < 0 || inst >= c->n_inst || !n_out) return fail(SDPD_E_INVALID, "bad argument");
    if (!c->cells_valid) return fail(SDPD_E_STATE, "no neighbour build for the current positions");
    CUDA_TRY(cudaDeviceSynchronize());
    const long long N = c->N;
    std::vector<int> cnt(N), perm(N), pinst(N);
    CUDA_TRY(cudaMemcpy(cnt.data(), c->b.ncnt, sizeof(int) * N, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(perm.data(), c->b.perm, sizeof(int) * N, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(pinst.data(), c->b.pinst, sizeof(int) * N, cudaMemcpyDeviceToHost));
    int kmax = 0;
    for (long long s = 0; s < N; ++s) kmax = std::max(kmax, cnt[s]);
    std::vector<int> nb((size_t)kmax * c->Npad);
    std::vector<uint8_t> fl((size_t)kmax * c->Npad);
    if (kmax) {
        // entries of the (skin) list within h at the current positions
        uint8_t *dfl = nullptr;
        CUDA_TRY(cudaMalloc(&dfl, (size_t)c->cap * c->Npad));
        launch_mark_pairs(c->b, dfl, 0);
        cudaError_t e1 = cudaMemcpy(fl.data(), dfl, fl.size(), cudaMemcpyDeviceToHost);
        cudaFree(dfl);
        if (e1 != cudaSuccess) return fail(SDPD_E_CUDA, "cudaMemcpy pair flags");
        CUDA_TRY(cudaMemcpy(nb.data(), c->b.nbr, sizeof(int) * nb.size(), cudaMemcpyDeviceToHost));
    }
    const long long o = c->hi[inst].begin;
    long long k = 0;
    for (long long s = 0; s < N; ++s) {
        const int gi = perm[s];
        if (pinst[gi] != inst) continue;
        for (int q = 0; q < cnt[s]; ++q) {
            const uint32_t e = (uint32_t)nb[(size_t)q * c->Npad + s];
            if ((e & NB_FAR) || !fl[(size_t)q * c->Npad + s]) continue;
            const int gj = perm[e];
            if (gj <= gi) continue;
            if (k < cap && ij) {
                ij[2 * k] = (int)(gi - o);
                ij[2 * k + 1] = (int)(gj - o);
            }
            ++k;
        }
    }
    *n_out = k;
    return check_err(c);
}

sdpd_status sdpd_count_pairs(sdpd_ctx *c, long long *n_pairs)
{
    if (!c || !n_pairs) return fail(SDPD_E_INVALID, "bad argument");
    if (!c->cells_valid) return fail(SDPD_E_STATE, "no neighbour build for the current positions");
    launch_count_pairs(c->b, 0);
    unsigned long long h = 0;
    CUDA_TRY(cudaMemcpy(&h, c->b.pair_count, sizeof(h), cudaMemcpyDeviceToHost));
    *n_pairs = (long long)h;
    return check_err(c);
}

sdpd_status sdpd_noise_normals(int precision, unsigned long long seed, int inst, unsigned step, long long n,
                               const unsigned *gi, const unsigned *gj, double *z_out)
{
    if (n < 0 || (n && (!gi || !gj || !z_out)) || inst < 0 ||
        (precision != SDPD_PREC_FP64 && precision != SDPD_PREC_SPLIT))
        return fail(SDPD_E_INVALID, "sdpd_noise_normals: bad argument");
    if (!n) return SDPD_OK;
    (void)cudaGetLastError();
    uint32_t *dg = nullptr;
    double *dz = nullptr;
    if (cudaMalloc(&dg, 2 * n * sizeof(uint32_t)) != cudaSuccess || cudaMalloc(&dz, 6 * n * sizeof(double)) != cudaSuccess) {
        cudaFree(dg);
        return fail(SDPD_E_OOM, "sdpd_noise_normals: cudaMalloc");
    }
    sdpd_status s = SDPD_OK;
    if (cudaMemcpy(dg, gi, n * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dg + n, gj, n * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess)
        s = fail(SDPD_E_CUDA, "sdpd_noise_normals: copy in");
    if (s == SDPD_OK) {
        const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFull), k1 = (uint32_t)(seed >> 32) ^ (uint32_t)inst;
        launch_noise_normals(precision, n, dg, dg + n, step, k0, k1, dz, 0);
        if (cudaMemcpy(z_out, dz, 6 * n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            s = fail(SDPD_E_CUDA, "sdpd_noise_normals: kernel or copy out");
    }
    cudaFree(dg);
    cudaFree(dz);
    return s;
}

sdpd_status sdpd_philox4x32_10(long long n, const unsigned *ctr, const unsigned *key, unsigned *out)
{
    if (n < 0 || (n && (!ctr || !key || !out))) return fail(SDPD_E_INVALID, "sdpd_philox4x32_10: bad argument");
    if (!n) return SDPD_OK;
    (void)cudaGetLastError();
    uint32_t *d = nullptr;
    if (cudaMalloc(&d, 10 * n * sizeof(uint32_t)) != cudaSuccess)
        return fail(SDPD_E_OOM, "sdpd_philox4x32_10: cudaMalloc");
    sdpd_status s = SDPD_OK;
    if (cudaMemcpy(d, ctr, 4 * n * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d + 4 * n, key, 2 * n * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess)
        s = fail(SDPD_E_CUDA, "sdpd_philox4x32_10: copy in");
    if (s == SDPD_OK) {
        launch_philox_raw(n, d, d + 4 * n, d + 6 * n, 0);
        if (cudaMemcpy(out, d + 6 * n, 4 * n * sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
            s = fail(SDPD_E_CUDA, "sdpd_philox4x32_10: kernel or copy out");
    }
    cudaFree(d);
    return s;
}

sdpd_status sdpd_diagnostics(sdpd_ctx *c, int inst, double out[16])
{
    if (!c || inst < 0 || inst >= c->n_inst || !out) return fail(SDPD_E_INVALID, "bad argument");
    sdpd_status s = ensure_geometry(c);
    if (s != SDPD_OK) return s;
    CUDA_TRY(cudaDeviceSynchronize());
    launch_diag(c->b, inst, 0, c->hi[inst].n);
    double h[16];
    CUDA_TRY(cudaMemcpy(h, c->b.probe, sizeof(h), cudaMemcpyDeviceToHost));
    for (int k = 0; k < 16; ++k) out[k] = 0.0;
    out[0] = h[0]; out[1] = h[1]; out[2] = h[2];
    out[3] = 0.5 * h[3];
    const double M = h[4], n = h[5];
    const double P2 = h[0] * h[0] + h[1] * h[1] + h[2] * h[2];
    out[4] = n > 0 ? (h[3] - (M > 0 ? P2 / M : 0.0)) / (3.0 * n) : 0.0;
    out[5] = h[6];
    out[6] = h[7];
    out[7] = h[8];
    out[8] = h[9];
    return check_err(c);
}

}  // extern "C"
