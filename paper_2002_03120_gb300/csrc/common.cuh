// common.cuh -- device data layout and helpers of libsdpd (sm_103a).
//
// Layout in HBM (one context, all instances concatenated):
//   master state, gid order  : x, v, w, F, T (double [N][3]); type, inst (int);
//                              mass props (double); rigid index maps
//   cell tables              : per-instance grids, Morton-ranked cell keys,
//                              cell counts / starts (counting sort)
//   sorted mirrors, slot order (rebuilt by each neighbour build):
//     split precision : A32 {x,y,z relative to own cell, bits(type|cell)}
//                       B32 {v, R}   C32 {w, m}   D32 {p/d^2, 1/d, 1/sqrt d, gid}
//     fp64            : A64 {x,y,z absolute, -} B64 C64 D64 likewise in double
//   neighbour list, column-major nbr[k * Npad + slot] (coalesced per warp)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sdpd.h"

namespace sdpd {

constexpr int T_FLUID = 0, T_RIGID = 1, T_INNER = 2, T_OUTER = 3;
constexpr double PI = 3.14159265358979323846;

// device error word bits
constexpr int ERR_NBR_CAP = 1, ERR_CELL_CAP = 2, ERR_CONTACT_CAP = 4, ERR_NONFINITE = 8,
              ERR_DOMAIN = 16, ERR_PAIR_CAP = 32, ERR_REV = 64;

// rigid-pair list entries beyond h (contact only) carry this flag
constexpr uint32_t NB_FAR = 0x80000000u;

// neighbour-cell table: up to 5 x 5 x 5 cells per cell (half-size cells),
// entries (key << 7) | ((ox + 2) + 5 (oy + 2) + 25 (oz + 2)), -1 = none
constexpr int ADJ = 125;
constexpr int PLANE_BASE = -16;   // contact-history partner codes of wall planes

// Per-instance constants, derived on the host from sdpd_params.
struct Inst {
    double origin[3], box[3], lo[3], cs[3], inv_cs[3];
    int nc[3], periodic[3];
    int sub;                   // cells per minimum cell width (1 or 2): the stencil reaches +-sub cells
    int cell_base, ncell;
    long long p_begin, p_end;
    double dx, rc, rc2, inv_rc, dt, hdt, isqrt_dt;
    double Wc, Fc, W0, Cn, mf, inv_dx3;
    double rho0, p0, alpha, beta_p;
    double Ca, Cb, eta, kBT, Ka, Kb;
    double coeff_c, coeff_d, coeff_r, coeff_t;
    double g[3], body_amp;
    int body_axis, split_axis;
    int filter, clamp, artvis, dem_law, noise, reinit;
    int alpha_int;             // alpha when it is an integer in [1, 32], else 0
    double artvis_rlim, artvis_e;
    double kn, kt_ratio, zeta, nu_p, E_p, mu_fric;
    double lub_gap_min, eps_min, Vf;
    double lever_fluid;
    uint32_t key0, key1;
    // float copies for the split-precision pair kernels
    float rcf, inv_rcf, csf[3], Wcf, Fcf, Caf, Cbf, Kaf, Kbf, isqrt_dtf;
    float coeff_cf, coeff_df, coeff_rf, coeff_tf, W0f, lever_fluidf;
    float guard_lo, guard_hi;   // r^2 band re-decided exactly in double
    float artvis_r2f_hi;        // collision pass: float prefilter bound
    // Verlet skin: lists hold pairs within rb = h (1 + skin); they stay valid
    // until a particle has moved skin h / 2 since the build
    double rb, rb2, half_skin;
    float rb2f;
    // the update kernel's bounds: origin + box (as the oracle forms it) and
    // the bits of box / 2, compared on the integer pipe
    double dom_hi[3];
    unsigned long long hbox_bits[3];
};

// Device buffers of a context (all device pointers).
struct Bufs {
    long long N, Npad;
    int n_inst, ncell_total, nrigid, cap, K;
    int pair_block;            // threads per block of the pair kernels (64, 128 or 256)
    int tpp;                   // lanes per particle of the direct force pass (1, 2 or 4)
    int cell_sub;              // cells per minimum cell width (1 or 2): picks the list kernel
    const Inst *inst;          // [n_inst]
    // master state (gid order)
    double *x, *v, *w, *F, *T;
    int *type, *pinst;
    double *R, *m, *Iner;               // radius, mass, moment of inertia
    int *rigid_of;             // gid -> rigid index or -1
    int *rigid_gid;            // rigid index -> gid
    // cells
    const int *cell_rank;      // [ncell_total] linear cell -> Morton rank (within instance)
    const int *cell_adj;       // [ncell_total][ADJ] (key << 7 | offset code), ascending key, -1 = none
    int *key, *slot_in_cell, *ccount, *cstart, *tmp_perm, *perm, *slot_of;
    int *scan_partials;        // [ceil(ncell_total/1024)+1]
    // mirrors
    float4 *A32, *B32, *C32, *D32;
    double4_32a *A64, *B64, *C64, *D64;
    int *stype;
    double *sd, *sp, *sp2;     // density, pressure (raw / filtered) per slot
    double *sdr;               // reinitialised density (scratch of the reinitialisation pass)
    double *xs;                // [N][3] staging of uploaded positions
    // neighbour lists: owned pairs first (Newton-3 ownership), see k_neighbors
    int *nbr, *ncnt, *nfirst;  // nfirst = length of the owned prefix
    int *skey;                 // cell key per slot
    uint16_t *rev;             // owned entry k of s -> row of the partner's column that
                               // receives s's result of the pair (its non-owned entry - nfirst);
                               // non-owned entry k of s -> position of s in the partner's list
    uint8_t *nbflag;           // per slot: bit 0 = has a rigid neighbour
    int capown;                // owned entries per particle in the pair buffer
    double *rm, *rI;           // [N] 1/m and 1/I rounded to nearest (the update divides with them)
    uint8_t *aclose;           // [N] slot has a mobile neighbour within the collision radius
    int *aclose_ok;            // the marks belong to the current positions and list
    void *resA, *resB;         // pair results [capown][Npad]: FP64 R4 {f, h.x}, R2 {h.y, h.z}
                               // (h = e x o) in the column of the particle that does not own
                               // the pair, row = its non-owned entry - nfirst; split float4
                               // {o, ce} in the owner's column at the owned entry, resB unused
    void *ownA, *ownB;         // per slot sums of the owned pairs
    // fluid-particle interaction per rigid index
    double *eps, *fdg;         // eps [nr], drag [nr][3]
    double *dsum;              // [nr][5] fluid sums of the drag: rigid volume, S, U
    double4_32a *rxn;              // per slot: F^DG / S_s (rigid slots only)
    float4 *rxn32;                 // the same in FP32 (split-precision pair kernels)
    // DEM history: old / new tables [nr][K]
    int *h_n, *h_part, *hn_n, *hn_part;
    double *h_del, *hn_del;
    // artificial viscosity scratch
    double *dv;
    // list reuse: exact cell-relative coordinates and displacement since the
    // last build (slot order); build gate and epochs; cached random normals
    double4_32a *xl64, *dsp;
    int *need_build;           // set by the drift when a particle moved half the skin
    unsigned *list_epoch;      // incremented by every build
    unsigned *cache_epoch;     // list epoch of the cached normals
    long long *cache_step;     // step of the cached normals
    void *zA, *zB;             // normals [capown][Npad]: R4 {z0..z3}, R2 {z4, z5}
    void *zdA, *zdB;           // direct pass: normals of every entry [cap][Npad] (same arena)
    int use_cache;
    int *fresh;                // a build happened since the last density
    // counters
    long long *step;
    int *err;
    unsigned long long *pair_count;
    unsigned long long *work;  // slot counter of the persistent pair kernels
    double *probe;             // scratch for probe / diagnostics
};

// ---------------------------------------------------------------- helpers
__host__ __device__ inline uint32_t morton_spread(uint32_t v)
{
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__host__ __device__ inline uint32_t pack_cell(int type, int cx, int cy, int cz)
{
    return (uint32_t)type | ((uint32_t)cx << 2) | ((uint32_t)cy << 12) | ((uint32_t)cz << 22);
}

__device__ __forceinline__ int unpack_type(uint32_t b) { return (int)(b & 3u); }
__device__ __forceinline__ int unpack_cx(uint32_t b) { return (int)((b >> 2) & 0x3FFu); }
__device__ __forceinline__ int unpack_cy(uint32_t b) { return (int)((b >> 12) & 0x3FFu); }
__device__ __forceinline__ int unpack_cz(uint32_t b) { return (int)((b >> 22) & 0x3FFu); }

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the
// multiply-xor S-box on a 128-bit counter with a Weyl-sequence key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a = c.x, b = c.z;
        const uint32_t hi0 = __umulhi(0xD2511F53u, a), lo0 = 0xD2511F53u * a;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, b), lo1 = 0xCD9E8D57u * b;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Six standard normals of the pair {gi, gj} at `step`: two Philox blocks,
// uniforms ((u >> 9) + 1/2) 2^-23 (exact in float and double), Box-Muller on
// (u0,u1), (u2,u3), (u4,u5) in precision R.  Scalars only (no local arrays).
// Table-driven FP64 pieces of the Box-Muller transform.  A uniform is
// U = ((u >> 9) + 1/2) 2^-23 = w 2^-24 with w = 2 (u >> 9) + 1 odd and below
// 2^24, so both the logarithm and the angle are taken from the integer w:
//  * ln U (Tang's table-driven logarithm, ACM TOMS 16, 1990): w = 2^e f,
//    f in [1, 2); c = 1 + j/128 from the top seven bits of f; f - c exact;
//    ln U = (e - 24) ln 2 + ln c + log1p((f - c)/c), the series to r^7
//    (r < 2^-7, truncation below 2^-59);
//  * sin, cos of 2 pi w 2^-24: quadrant from the top two bits of w, the
//    remaining angle split as (pi/2)(h/256) + t, h the next eight bits and
//    t < (pi/2)/256, Taylor series of sin t (to t^5) and cos t (to t^6), and
//    the angle-addition formulas.
// Both are accurate to a few units in the last place.
#include "bm_tables.cuh"

__device__ __forceinline__ double bm_log_w(uint32_t w)
{
    const int e = 31 - __clz(w);
    const uint64_t frac = e ? ((uint64_t)(w ^ (1u << e))) << (52 - e) : 0ull;
    const int j = (int)(frac >> 45);
    const double f = __longlong_as_double((long long)(0x3FF0000000000000ull | frac));
    const double c = __longlong_as_double((long long)(0x3FF0000000000000ull | ((uint64_t)j << 45)));
    const double2 t = __ldg(&BM_LOG_TAB[j]);
    const double r = (f - c) * t.y;
    double p = fma(r, 1.0 / 7.0, -1.0 / 6.0);
    p = fma(p, r, 1.0 / 5.0);
    p = fma(p, r, -0.25);
    p = fma(p, r, 1.0 / 3.0);
    p = fma(p, r, -0.5);
    p = fma(p, r, 1.0);
    return (__ldg(&BM_LOG_E[e]) + t.x) + p * r;
}

__device__ __forceinline__ void bm_sincos_w(uint32_t w, double &s, double &c)
{
    const uint32_t q = w >> 22, h = (w >> 14) & 255u, lo = w & 16383u;
    const double lod = __longlong_as_double((long long)(0x4330000000000000ull | lo)) - 4503599627370496.0;
    const double t = lod * (1.5707963267948966 / 4194304.0);
    const double t2 = t * t;
    const double sl = t * fma(t2, fma(t2, 1.0 / 120.0, -1.0 / 6.0), 1.0);
    const double cl = fma(t2, fma(t2, fma(t2, -1.0 / 720.0, 1.0 / 24.0), -0.5), 1.0);
    const double2 sc = __ldg(&BM_SC_TAB[h]);
    const double sa = fma(sc.x, cl, sc.y * sl);
    const double ca = fma(sc.y, cl, -(sc.x * sl));
    // quadrant: swap and sign flips on the bit patterns (integer pipe)
    const unsigned long long SIGN = 0x8000000000000000ull;
    const unsigned long long fs = (q & 2) ? SIGN : 0ull, fc = ((q + 1) & 2) ? SIGN : 0ull;
    s = __longlong_as_double((long long)((unsigned long long)__double_as_longlong((q & 1) ? ca : sa) ^ fs));
    c = __longlong_as_double((long long)((unsigned long long)__double_as_longlong((q & 1) ? sa : ca) ^ fc));
}

template <class R> struct BoxMuller;
template <> struct BoxMuller<double> {
    __device__ __forceinline__ static void pair(uint32_t ua, uint32_t ub, double &z0, double &z1)
    {
        const double rad = sqrt(-2.0 * bm_log_w(((ua >> 9) << 1) | 1u));
        double s, c;
        bm_sincos_w(((ub >> 9) << 1) | 1u, s, c);
        // rounded products: no later sum fuses them, so a normal read back
        // from the cache and one drawn here enter the force identically
        z0 = __dmul_rn(rad, c);
        z1 = __dmul_rn(rad, s);
    }
};
// ln U of a uniform U = (m + 1/2) 2^-23 in FP32, from the hardware base-2
// logarithm (absolute error about 2^-22 on [2^-24, 1)) where |ln U| >= 1/64,
// and from the Taylor series of ln(1 - d) in the exact d = 1 - U below that,
// where an absolute error would swamp the small logarithm: five terms leave
// a truncation below d^6 / 6 < 2^-38.  The result carries a relative error
// of a few 1e-7 at most over the whole range.
__device__ __forceinline__ float bm_log_f32(float U)
{
    const float d = 1.0f - U;   // exact: U has at most 24 significant bits
    const float ser = -d * fmaf(d, fmaf(d, fmaf(d, fmaf(d, 0.2f, 0.25f), 1.0f / 3.0f), 0.5f), 1.0f);
    const float hw = __log2f(U) * 0.69314718055994531f;
    return d < 0.015625f ? ser : hw;
}

// FP32: the logarithm above (ln U1 -> 0 as U1 -> 1, where an absolute error
// would swamp it), the radius as x rsqrt(x), and the angle
// 2 pi U2 = pi + 2 pi (U2 - 1/2) through the hardware sine and cosine on
// [-pi, pi] (absolute error below 2^-21.4; cos(pi + t) = -cos t exactly).  A
// normal is within about 5e-6 of the exact value (radius up to 5.8).
template <> struct BoxMuller<float> {
    __device__ __forceinline__ static void pair(uint32_t ua, uint32_t ub, float &z0, float &z1)
    {
        const float U1 = ((float)(ua >> 9) + 0.5f) * (1.0f / 8388608.0f);
        const float U2 = ((float)(ub >> 9) + 0.5f) * (1.0f / 8388608.0f);
        const float m2l = -2.0f * bm_log_f32(U1);   // > 0: U1 <= 1 - 2^-24
        const float rad = m2l * rsqrtf(m2l);
        float s, c;
        __sincosf(6.28318530717958648f * (U2 - 0.5f), &s, &c);
        z0 = __fmul_rn(rad, -c);
        z1 = __fmul_rn(rad, -s);
    }
};

template <class R>
__device__ __forceinline__ void pair_normals(uint32_t gi, uint32_t gj, uint32_t step, uint32_t k0,
                                             uint32_t k1, R &z0, R &z1, R &z2, R &z3, R &z4, R &z5)
{
    const uint32_t lo = min(gi, gj), hi = max(gi, gj);
    const uint4 a = philox4x32_10(make_uint4(lo, hi, step, 0u), k0, k1);
    const uint4 b = philox4x32_10(make_uint4(lo, hi, step, 1u), k0, k1);
    BoxMuller<R>::pair(a.x, a.y, z0, z1);
    BoxMuller<R>::pair(a.z, a.w, z2, z3);
    BoxMuller<R>::pair(b.x, b.y, z4, z5);
}

// Geometry constants of an instance held in registers for the pair loop.
template <class R> struct Geo;
template <> struct Geo<float> {
    int n0, n1, n2, dm;   // dm: the farthest neighbour cell of the stencil (1 or 2)
    float c0, c1, c2;
    float glo, ghi;   // r^2 guard band (copied: a store in a pair loop may not
                      // force them to be reloaded from the instance table)
    __device__ __forceinline__ explicit Geo(const Inst &I)
        : n0(I.nc[0]), n1(I.nc[1]), n2(I.nc[2]), dm(I.sub), c0(I.csf[0]), c1(I.csf[1]), c2(I.csf[2]),
          glo(I.guard_lo), ghi(I.guard_hi) {}
    __device__ __forceinline__ void disp(const float4 &Ai, const float4 &Aj, float &rx, float &ry,
                                         float &rz) const
    {
        const uint32_t bi = __float_as_uint(Ai.w), bj = __float_as_uint(Aj.w);
        int d0 = unpack_cx(bi) - unpack_cx(bj), d1 = unpack_cy(bi) - unpack_cy(bj),
            d2 = unpack_cz(bi) - unpack_cz(bj);
        // The cells are those of the list build, and a listed pair was at
        // most dm cells apart then.  A periodic axis holds at least 2 dm + 1
        // cells, so a larger difference is a wrap.  On a closed axis the
        // difference never exceeds dm, so the same test needs no flag.
        d0 = d0 > dm ? d0 - n0 : (d0 < -dm ? d0 + n0 : d0);
        d1 = d1 > dm ? d1 - n1 : (d1 < -dm ? d1 + n1 : d1);
        d2 = d2 > dm ? d2 - n2 : (d2 < -dm ? d2 + n2 : d2);
        rx = (Ai.x - Aj.x) + (float)d0 * c0;
        ry = (Ai.y - Aj.y) + (float)d1 * c1;
        rz = (Ai.z - Aj.z) + (float)d2 * c2;
    }
};
// |x| compared through the IEEE bit patterns, which order like the values
// for non-negative numbers: an exact test that runs on the integer pipe and
// leaves the FP64 pipe (the bound of the FP64 pair kernels) to arithmetic.
__device__ __forceinline__ unsigned long long abs_bits(double x)
{
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

template <> struct Geo<double> {
    bool p0, p1, p2;
    double L0, L1, L2;
    unsigned long long h0, h1, h2;   // bits of L/2
    double rc2;                      // h^2 (copied, as the guard band of the FP32 form)
    __device__ __forceinline__ explicit Geo(const Inst &I)
        : p0(I.periodic[0]), p1(I.periodic[1]), p2(I.periodic[2]), L0(I.box[0]), L1(I.box[1]),
          L2(I.box[2]), h0(abs_bits(0.5 * I.box[0])), h1(abs_bits(0.5 * I.box[1])),
          h2(abs_bits(0.5 * I.box[2])), rc2(I.rc2) {}
    // minimum image: d - L if d > L/2, d + L if d < -L/2 (the same operations
    // as the oracle; the rare wrap is a branch)
    __device__ __forceinline__ static double img(double d, bool p, double L, unsigned long long hb)
    {
        if (p && abs_bits(d) > hb) d = d > 0.0 ? d - L : d + L;
        return d;
    }
    __device__ __forceinline__ void disp(const double4_32a &Ai, const double4_32a &Aj, double &rx,
                                         double &ry, double &rz) const
    {
        rx = img(Ai.x - Aj.x, p0, L0, h0);
        ry = img(Ai.y - Aj.y, p1, L1, h1);
        rz = img(Ai.z - Aj.z, p2, L2, h2);
    }
};

// Warp sum (butterfly: every lane ends with the same, order-fixed result).
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The oracle's distance: r = x_i - x_j with the minimum image on periodic
// axes, r^2 = (x*x + y*y) + z*z, evaluated without fused multiply-adds.
__device__ __forceinline__ double exact_r2(const double *xi, const double *xj, const Inst &I)
{
    double d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double t = __dsub_rn(xi[a], xj[a]);
        if (I.periodic[a]) {
            const double hL = 0.5 * I.box[a];
            if (t > hL) t = __dsub_rn(t, I.box[a]);
            else if (t < -hL) t = __dadd_rn(t, I.box[a]);
        }
        d[a] = t;
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

// r_ij < h decided exactly from the FP64 master positions (gids gi, gj).
__device__ __forceinline__ bool exact_within(const Bufs &b, const Inst &I, int gi, int gj)
{
    const double xi[3] = { b.x[3 * gi], b.x[3 * gi + 1], b.x[3 * gi + 2] };
    const double xj[3] = { b.x[3 * gj], b.x[3 * gj + 1], b.x[3 * gj + 2] };
    return exact_r2(xi, xj, I) < I.rc2;
}

// message returned by sdpd_last_error() on this thread (defined in api.cu)
void set_last_error(const char *msg);

// ---------------------------------------------------------------- launchers
// (defined in k_cells.cu, k_pairs.cu, k_update.cu; all enqueue on `st`)
// gate: nullptr = always build; else build only when *gate != 0
void launch_build(const Bufs &b, int precision, int need_rev, const int *gate, cudaStream_t st);
// dflags: bit 0 some instance filters the pressure, bit 1 some instance
// reinitialises the density, bit 2 some instance has the artificial viscosity
// (the density pass then marks the collision candidates)
void launch_density(const Bufs &b, int precision, int dflags, int newton3, const int *gate, cudaStream_t st);
void launch_drag(const Bufs &b, int precision, cudaStream_t st);
// force mode: 0 direct, 1 Newton 3 (half pairs + gather), 2 pair stream
void launch_forces(const Bufs &b, int precision, int velver, int newton3, cudaStream_t st);
void init_pair_kernels();
void init_cell_kernels();
void launch_mark_pairs(const Bufs &b, uint8_t *flags, cudaStream_t st);
void launch_integrate(const Bufs &b, int precision, int velver, int any_artvis, cudaStream_t st);
void launch_step_done(const Bufs &b, cudaStream_t st);
void launch_probe(const Bufs &b, int inst, int nbins, cudaStream_t st, long long n);
void launch_diag(const Bufs &b, int inst, cudaStream_t st, long long n);
void launch_count_pairs(const Bufs &b, cudaStream_t st);
void launch_absorb(const Bufs &b, int precision, const double *xs, int has_x, cudaStream_t st);
void launch_philox_raw(long long n, const uint32_t *ctr, const uint32_t *key, uint32_t *out, cudaStream_t st);
void launch_noise_normals(int precision, long long n, const uint32_t *gi, const uint32_t *gj, uint32_t step,
                          uint32_t k0, uint32_t k1, double *out, cudaStream_t st);

}  // namespace sdpd
