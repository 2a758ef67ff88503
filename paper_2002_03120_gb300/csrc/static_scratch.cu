// static_scratch.cu -- sdpd_density_noalloc: number density and pressure of
// one particle set without any device allocation.
//
// Some callers cannot let a library allocate device memory: applications
// whose allocator (for example a framework's caching allocator) owns the
// whole device and forbids foreign cudaMalloc calls, and control loops that
// cannot afford the implicit device-wide synchronisation cudaMalloc and
// cudaFree may cause.  This entry point serves them: its scratch (cell keys,
// slots, counts, starts and the particle permutation) lives in one file-scope
// __device__ array of fixed size that every GPU loading the library keeps
// until process exit; the caller passes only inputs and outputs.
//
// The paper has no counterpart of this entry point; it computes the same
// quantities as sdpd_build_cells + sdpd_compute_density (Eqs. compdens and
// prtcpres with the kernel normalisation and the optional clamp) for FP64
// positions, without the pressure filter.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "common.cuh"

namespace sdpd {
namespace noalloc {

constexpr int NMAX = SDPD_NOALLOC_MAX_PARTICLES;
constexpr int CMAX = SDPD_NOALLOC_MAX_CELLS;
// layout of the scratch array (ints): key[NMAX] | slot[NMAX] | perm[NMAX] |
// count[CMAX] | start[CMAX + 1]
constexpr size_t OFF_KEY = 0, OFF_SLOT = NMAX, OFF_PERM = 2 * (size_t)NMAX,
                 OFF_COUNT = 3 * (size_t)NMAX, OFF_START = 3 * (size_t)NMAX + CMAX,
                 SCRATCH_INTS = 3 * (size_t)NMAX + 2 * (size_t)CMAX + 1;

static __device__ __align__(256) int g_scratch[SCRATCH_INTS];

struct Grid {
    double lo[3], cs[3], inv_cs[3], box[3];
    int nc[3], periodic[3];
    double rc, rc2, Wc, Cn, mf, inv_dx3, rho0, p0, alpha, beta_p;
    int clamp;
    long long n;
};

// A periodic coordinate folded into [lo, lo + box): the identity for a
// coordinate already inside (x - 0 * box = x exactly), so in-box inputs give
// the same displacements as the context path.
__device__ __forceinline__ double wrap_of(double x, const Grid &G, int a)
{
    if (!G.periodic[a]) return x;
    return x - G.box[a] * floor((x - G.lo[a]) / G.box[a]);
}

// Cell coordinate of a (wrapped) coordinate, clamped into the grid in double
// before the conversion, so that a huge or non-finite value cannot index
// outside it.  On wall axes the clamp is monotone, so two particles closer
// than r_c still fall into the same or adjacent cells.
__device__ __forceinline__ int cell_of(double x, const Grid &G, int a)
{
    const double f = floor((x - G.lo[a]) * G.inv_cs[a]);
    if (!(f >= 0.0)) return 0;   // negative or NaN
    if (f >= (double)(G.nc[a] - 1)) return G.nc[a] - 1;
    return (int)f;
}

__device__ __forceinline__ bool finite3(const double *x)
{
    return isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]);
}

__global__ void k_na_clear(int *scr, int ncell)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell) scr[OFF_COUNT + c] = 0;
}

__global__ void k_na_count(int *scr, Grid G, const double *x)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G.n) return;
    const int cx = cell_of(wrap_of(x[3 * i], G, 0), G, 0), cy = cell_of(wrap_of(x[3 * i + 1], G, 1), G, 1),
              cz = cell_of(wrap_of(x[3 * i + 2], G, 2), G, 2);
    const int key = (cz * G.nc[1] + cy) * G.nc[0] + cx;
    scr[OFF_KEY + i] = key;
    scr[OFF_SLOT + i] = atomicAdd(&scr[OFF_COUNT + key], 1);
}

// one block of 1024 threads: exclusive scan of the cell counts
__global__ void k_na_scan(int *scr, int ncell, long long n)
{
    __shared__ int part[1024];
    const int per = (ncell + 1023) / 1024;
    const int b0 = threadIdx.x * per;
    int sum = 0;
    for (int c = b0; c < b0 + per && c < ncell; ++c) sum += scr[OFF_COUNT + c];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int c = b0; c < b0 + per && c < ncell; ++c) {
        scr[OFF_START + c] = run;
        run += scr[OFF_COUNT + c];
    }
    if (threadIdx.x == 0) scr[OFF_START + ncell] = (int)n;
}

__global__ void k_na_scatter(int *scr, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    scr[OFF_PERM + scr[OFF_START + scr[OFF_KEY + i]] + scr[OFF_SLOT + i]] = (int)i;
}

__global__ void k_na_density(const int *scr, Grid G, const double *x, const int *type, double *d_out,
                             double *p_out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G.n) return;
    const double xr[3] = { x[3 * i], x[3 * i + 1], x[3 * i + 2] };
    if (!finite3(xr)) {
        // no density for a particle without a position; it is nobody's
        // neighbour either (every comparison with NaN fails)
        d_out[i] = NAN;
        p_out[i] = NAN;
        return;
    }
    double d;
    if (type[i] == T_OUTER) {
        d = G.inv_dx3;
    } else {
        const double xi[3] = { wrap_of(xr[0], G, 0), wrap_of(xr[1], G, 1), wrap_of(xr[2], G, 2) };
        const int ci[3] = { cell_of(xi[0], G, 0), cell_of(xi[1], G, 1), cell_of(xi[2], G, 2) };
        double sum = G.Wc;  // self term W(0)
        for (int oz = -1; oz <= 1; ++oz) {
            int cz = ci[2] + oz;
            if (G.periodic[2]) cz = (cz + G.nc[2]) % G.nc[2];
            else if (cz < 0 || cz >= G.nc[2]) continue;
            for (int oy = -1; oy <= 1; ++oy) {
                int cy = ci[1] + oy;
                if (G.periodic[1]) cy = (cy + G.nc[1]) % G.nc[1];
                else if (cy < 0 || cy >= G.nc[1]) continue;
                for (int ox = -1; ox <= 1; ++ox) {
                    int cx = ci[0] + ox;
                    if (G.periodic[0]) cx = (cx + G.nc[0]) % G.nc[0];
                    else if (cx < 0 || cx >= G.nc[0]) continue;
                    const int key = (cz * G.nc[1] + cy) * G.nc[0] + cx;
                    for (int q = scr[OFF_START + key]; q < scr[OFF_START + key + 1]; ++q) {
                        const int j = scr[OFF_PERM + q];
                        if (j == i) continue;
                        double r[3];
                        for (int a = 0; a < 3; ++a) {
                            double t = __dsub_rn(xi[a], wrap_of(x[3 * (long long)j + a], G, a));
                            if (G.periodic[a]) {
                                const double hL = 0.5 * G.box[a];
                                if (t > hL) t = __dsub_rn(t, G.box[a]);
                                else if (t < -hL) t = __dadd_rn(t, G.box[a]);
                            }
                            r[a] = t;
                        }
                        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(r[0], r[0]), __dmul_rn(r[1], r[1])),
                                                    __dmul_rn(r[2], r[2]));
                        if (!(r2 < G.rc2)) continue;
                        const double q1 = sqrt(r2) / G.rc, om = 1.0 - q1;
                        sum += G.Wc * (1.0 + 3.0 * q1) * om * om * om;
                    }
                }
            }
        }
        d = G.Cn * sum;
    }
    double p = G.p0 * pow(G.mf * d / G.rho0, G.alpha) - G.beta_p;
    if (G.clamp && p < 0.0) p = 0.0;
    d_out[i] = d;
    p_out[i] = p;
}

// Device address of the scratch array, resolved once per device (with that
// device current) on the first call made on it and kept for the process.  A
// device reset (cudaDeviceReset, or another library resetting the primary
// context) reloads the module and may move the array, so the library must
// not be used across one.
std::mutex g_mu;
int *g_addr[64] = { nullptr };

}  // namespace noalloc
}  // namespace sdpd

namespace {
struct NaErr {
    void operator=(const std::string &m) { sdpd::set_last_error(m.c_str()); }
} g_na_err;

double na_W(double r, double h)
{
    if (r >= h) return 0.0;
    const double q = r / h, om = 1.0 - q;
    return 105.0 / (16.0 * sdpd::PI * h * h * h) * (1.0 + 3.0 * q) * om * om * om;
}
}  // namespace

extern "C" sdpd_status sdpd_density_noalloc(const sdpd_params *p, long long n, const double *x,
                                            const int *type, double *d_out, double *p_out,
                                            void *stream)
{
    using namespace sdpd::noalloc;
    if (!p || n < 0 || (n && (!x || !type || !d_out || !p_out))) {
        g_na_err = "sdpd_density_noalloc: NULL argument or negative count";
        return SDPD_E_INVALID;
    }
    if (n > NMAX) {
        g_na_err = "sdpd_density_noalloc: " + std::to_string(n) + " particles exceed the static scratch limit of " +
                   std::to_string(NMAX);
        return SDPD_E_INVALID;
    }
    if (!(p->dx > 0) || !(p->r_c > 0) || !(p->rho0 > 0)) {
        g_na_err = "sdpd_density_noalloc: dx, r_c, rho0 must be > 0";
        return SDPD_E_INVALID;
    }
    // the kernel normalisation sums W over a lattice of (2 ceil(r_c/dx) + 3)^3
    // sites on the host
    if (!(p->r_c / p->dx <= 32.0)) {
        g_na_err = "sdpd_density_noalloc: r_c / dx must be finite and at most 32";
        return SDPD_E_INVALID;
    }
    Grid G{};
    // every axis: a finite origin, a finite box > 0 and a finite number of
    // cells in [1, CMAX] decided in double before any integer conversion,
    // so that no product of cell counts can overflow or turn negative
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(p->origin[a]) || !std::isfinite(p->box[a]) || !(p->box[a] > 0.0) ||
            !std::isfinite(p->r_c) || !std::isfinite(p->dx)) {
            g_na_err = "sdpd_density_noalloc: origin, box, dx and r_c must be finite, box > 0 on every axis";
            return SDPD_E_INVALID;
        }
        G.box[a] = p->box[a];
        G.periodic[a] = p->periodic[a] ? 1 : 0;
        const double ncd = G.periodic[a] ? std::floor(p->box[a] / p->r_c)
                                         : std::ceil((p->box[a] + 4.0 * p->r_c) / p->r_c);
        if (!std::isfinite(ncd) || ncd < (G.periodic[a] ? 3.0 : 1.0)) {
            g_na_err = G.periodic[a] ? "sdpd_density_noalloc: periodic axis narrower than 3 r_c"
                                     : "sdpd_density_noalloc: box / r_c is not a finite positive cell count";
            return SDPD_E_INVALID;
        }
        if (ncd > (double)CMAX) {
            g_na_err = "sdpd_density_noalloc: " + std::to_string((long long)ncd) + " cells along axis " +
                       std::to_string(a) + " exceed the static scratch limit of " + std::to_string(CMAX);
            return SDPD_E_INVALID;
        }
        G.nc[a] = (int)ncd;
        if (G.periodic[a]) {
            G.cs[a] = p->box[a] / G.nc[a];
            G.lo[a] = p->origin[a];
        } else {
            // the fluid region plus two kernel radii of dummy-particle layers;
            // particles beyond are clamped into the boundary cells (still exact)
            G.cs[a] = p->r_c;
            G.lo[a] = p->origin[a] - 2.0 * p->r_c;
        }
        G.inv_cs[a] = 1.0 / G.cs[a];
    }
    const long long ncell = (long long)G.nc[0] * G.nc[1] * G.nc[2];   // each factor <= CMAX
    if (ncell > CMAX) {
        g_na_err = "sdpd_density_noalloc: " + std::to_string(ncell) + " cells exceed the static scratch limit of " +
                   std::to_string(CMAX);
        return SDPD_E_INVALID;
    }
    const double h = p->r_c;
    G.rc = h;
    G.rc2 = h * h;
    G.Wc = 105.0 / (16.0 * sdpd::PI * h * h * h);
    const int m = (int)std::ceil(h / p->dx) + 1;
    double lat = 0.0;
    for (int k = -m; k <= m; ++k)
        for (int j = -m; j <= m; ++j)
            for (int i = -m; i <= m; ++i) lat += na_W(std::sqrt((double)(i * i + j * j + k * k)) * p->dx, h);
    G.Cn = 1.0 / (p->dx * p->dx * p->dx * lat);
    G.mf = p->rho0 * p->dx * p->dx * p->dx;
    G.inv_dx3 = 1.0 / (p->dx * p->dx * p->dx);
    G.rho0 = p->rho0;
    G.p0 = p->p0;
    G.alpha = p->alpha;
    G.beta_p = p->beta_p;
    G.clamp = p->clamp_negative_p ? 1 : 0;
    G.n = n;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        g_na_err = "sdpd_density_noalloc: no current CUDA device";
        return SDPD_E_CUDA;
    }
    int *scr = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *ptr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
            if (e != cudaSuccess) {
                g_na_err = std::string("sdpd_density_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                return SDPD_E_CUDA;
            }
            g_addr[dev] = (int *)ptr;
        }
        scr = g_addr[dev];
    }
    if (n == 0) return SDPD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    (void)cudaGetLastError();
    const int nc_i = (int)ncell;
    k_na_clear<<<(nc_i + 255) / 256, 256, 0, st>>>(scr, nc_i);
    k_na_count<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(scr, G, x);
    k_na_scan<<<1, 1024, 0, st>>>(scr, nc_i, n);
    k_na_scatter<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(scr, n);
    k_na_density<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(scr, G, x, type, d_out, p_out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_na_err = std::string("sdpd_density_noalloc: launch: ") + cudaGetErrorString(e);
        return SDPD_E_CUDA;
    }
    return SDPD_OK;
}
