// k_pairs.cu -- the pair passes of one velocity-Verlet sub-step.
//
//   k_density      compute_particle_dens + compute_particle_pres (Eqs. compdens,
//                  prtcpres; kernel normalisation; negative-pressure clamp)
//   k_filter       smoothe_particle_pres (Shepard-weighted pressure)
//   k_drag         compute_fpi_action (Eqs. fvfdef, beta, F_fpi_DG)
//   k_force_half + k_force_gather (Newton-3) or k_force_fluid (direct):
//                  compute_fluid on fluid particles + compute_fpi_reaction
//                  (Eqs. FijC, FijD, FijR, FijT, F_fpi_DG_reac) + torque
//   k_force_rigid  compute_fluid on rigid particles (Eq. F_fpi_PG) +
//                  compute_rigid (Eqs. dem_fnij .. slideref, lubri), FP64
//
// Neighbour lists hold every pair within the build radius h (1 + skin); each
// pass decides r_ij < h exactly before using a pair (float test outside a
// +-1e-5 guard band, the oracle's double expression inside it, or the double
// expression directly in FP64 mode), so the pairs evaluated are exactly the
// paper's.  No atomics on forces: a thread writes only its own particle, and
// the Newton-3 pass hands each pair result to the partner through a buffer;
// every sum has a fixed order.  The random matrix of a pair is regenerated
// from the counter (min gid, max gid, step) or, in the second evaluation of a
// step, read back from the first one's cache (same counter, same bits).
#include <algorithm>
#include "common.cuh"

namespace sdpd {

template <class R> struct Vec;
template <> struct Vec<float> { using T4 = float4; };
template <> struct Vec<double> { using T4 = double4_32a; };
template <class R> struct Vec2;
template <> struct Vec2<float> { using T2 = float2; };
template <> struct Vec2<double> { using T2 = double2; };

// a < b for a, b >= 0: the value compare in FP32, the bit-pattern compare
// (same result, integer pipe) in FP64
__device__ __forceinline__ bool lt_nonneg(float a, float b) { return a < b; }
__device__ __forceinline__ bool lt_nonneg(double a, double b) { return abs_bits(a) < abs_bits(b); }

template <class R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ float rsqrt_<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_<double>(double x) { return rsqrt(x); }

template <class R> struct Mir;
template <> struct Mir<float> {
    __device__ __forceinline__ static const float4 *A(const Bufs &b) { return b.A32; }
    __device__ __forceinline__ static const float4 *B(const Bufs &b) { return b.B32; }
    __device__ __forceinline__ static const float4 *C(const Bufs &b) { return b.C32; }
    __device__ __forceinline__ static float4 *D(const Bufs &b) { return b.D32; }
};
template <> struct Mir<double> {
    __device__ __forceinline__ static const double4_32a *A(const Bufs &b) { return b.A64; }
    __device__ __forceinline__ static const double4_32a *B(const Bufs &b) { return b.B64; }
    __device__ __forceinline__ static const double4_32a *C(const Bufs &b) { return b.C64; }
    __device__ __forceinline__ static double4_32a *D(const Bufs &b) { return b.D64; }
};

__device__ __forceinline__ int mir_type(const float4 &A) { return unpack_type(__float_as_uint(A.w)); }
__device__ __forceinline__ int mir_type(const double4_32a &A) { return (int)A.w; }
__device__ __forceinline__ uint32_t mir_gid(const float4 &D) { return __float_as_uint(D.w); }
__device__ __forceinline__ uint32_t mir_gid(const double4_32a &D) { return (uint32_t)D.w; }
// The density terms of a particle for the pair routine.  FP32 records keep
// p/d^2 in B.w and 1/d in C.w, next to the velocity and the spin, so that a
// pass reading no gid (the second evaluation, normals from the cache) needs
// two records of a partner instead of three; 1/sqrt(d_i d_j) is then formed as
// sqrt(1/d_i 1/d_j).  FP64 records: D = {p/d^2, 1/d, 1/sqrt(d), gid}.
__device__ __forceinline__ float mir_pd2(const float4 &B, const float4 &) { return B.w; }
__device__ __forceinline__ double mir_pd2(const double4_32a &, const double4_32a &D) { return D.x; }
__device__ __forceinline__ float mir_invd(const float4 &C, const float4 &) { return C.w; }
__device__ __forceinline__ double mir_invd(const double4_32a &, const double4_32a &D) { return D.y; }
// om / sqrt(d_i d_j); FP32: x rsqrt(x) of x = 1/d_i 1/d_j > 0 (the hardware
// reciprocal square root, about 2 ulp, the same in every pass)
__device__ __forceinline__ float mir_rs(float om, const float4 &Ci, const float4 &, const float4 &Cj, const float4 &)
{
    const float x = Ci.w * Cj.w;
    return om * (x * rsqrtf(x));
}
__device__ __forceinline__ double mir_rs(double om, const double4_32a &, const double4_32a &Di, const double4_32a &,
                                         const double4_32a &Dj)
{
    return om * Di.z * Dj.z;
}

template <class R> struct K;  // kernel constants in precision R
template <> struct K<float> {
    __device__ __forceinline__ static float inv_rc(const Inst &I) { return I.inv_rcf; }
    __device__ __forceinline__ static float Wc(const Inst &I) { return I.Wcf; }
    __device__ __forceinline__ static float Fc(const Inst &I) { return I.Fcf; }
    __device__ __forceinline__ static float W0(const Inst &I) { return I.W0f; }
    __device__ __forceinline__ static float Ca(const Inst &I) { return I.Caf; }
    __device__ __forceinline__ static float Cb(const Inst &I) { return I.Cbf; }
    __device__ __forceinline__ static float Ka(const Inst &I) { return I.Kaf; }
    __device__ __forceinline__ static float Kb(const Inst &I) { return I.Kbf; }
    __device__ __forceinline__ static float isdt(const Inst &I) { return I.isqrt_dtf; }
    __device__ __forceinline__ static float cc(const Inst &I) { return I.coeff_cf; }
    __device__ __forceinline__ static float cd(const Inst &I) { return I.coeff_df; }
    __device__ __forceinline__ static float cr(const Inst &I) { return I.coeff_rf; }
    __device__ __forceinline__ static float ct(const Inst &I) { return I.coeff_tf; }
    __device__ __forceinline__ static float lever(const Inst &I) { return I.lever_fluidf; }
};
template <> struct K<double> {
    __device__ __forceinline__ static double inv_rc(const Inst &I) { return I.inv_rc; }
    __device__ __forceinline__ static double Wc(const Inst &I) { return I.Wc; }
    __device__ __forceinline__ static double Fc(const Inst &I) { return I.Fc; }
    __device__ __forceinline__ static double W0(const Inst &I) { return I.W0; }
    __device__ __forceinline__ static double Ca(const Inst &I) { return I.Ca; }
    __device__ __forceinline__ static double Cb(const Inst &I) { return I.Cb; }
    __device__ __forceinline__ static double Ka(const Inst &I) { return I.Ka; }
    __device__ __forceinline__ static double Kb(const Inst &I) { return I.Kb; }
    __device__ __forceinline__ static double isdt(const Inst &I) { return I.isqrt_dt; }
    __device__ __forceinline__ static double cc(const Inst &I) { return I.coeff_c; }
    __device__ __forceinline__ static double cd(const Inst &I) { return I.coeff_d; }
    __device__ __forceinline__ static double cr(const Inst &I) { return I.coeff_r; }
    __device__ __forceinline__ static double ct(const Inst &I) { return I.coeff_t; }
    __device__ __forceinline__ static double lever(const Inst &I) { return I.lever_fluid; }
};

// Displacement r_ij = r_i - r_j from the mirrors and the exact decision
// r_ij < h (gi: gid of i; j: slot of the partner, used only in the band).
template <class R> struct Rel;
template <> struct Rel<float> {
    __device__ __forceinline__ static bool get(const Bufs &b, const Inst &I, const Geo<float> &geo,
                                               const float4 &Ai, const float4 &Aj, int gi, int j,
                                               float &rx, float &ry, float &rz, float &r2)
    {
        geo.disp(Ai, Aj, rx, ry, rz);
        r2 = rx * rx + ry * ry + rz * rz;
        if (r2 < geo.glo) return true;
        if (r2 > geo.ghi) return false;
        return exact_within(b, I, gi, b.perm[j]);
    }
};
template <> struct Rel<double> {
    __device__ __forceinline__ static bool get(const Bufs &, const Inst &I, const Geo<double> &geo,
                                               const double4_32a &Ai, const double4_32a &Aj, int, int,
                                               double &rx, double &ry, double &rz, double &r2)
    {
        geo.disp(Ai, Aj, rx, ry, rz);
        r2 = __dadd_rn(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)), __dmul_rn(rz, rz));
        return abs_bits(r2) < abs_bits(geo.rc2);   // r2 >= 0: the bit order is the value order
    }
};

// Neumaier-compensated running sum (split precision density and filter).
struct KSum {
    float s, c;
    __device__ __forceinline__ void add(float v)
    {
        const float t = s + v;
        c += (fabsf(s) >= fabsf(v)) ? ((s - t) + v) : ((v - t) + s);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
template <class R> struct Acc;
template <> struct Acc<float> {
    KSum k;
    __device__ __forceinline__ explicit Acc(double v0) : k{ (float)v0, 0.f } {}
    __device__ __forceinline__ void add(float v) { k.add(v); }
    __device__ __forceinline__ double value() const { return k.value(); }
};
// The density sum: every term is W(q) <= W(0), and the sum starts at the
// self term W(0), so |s| >= |v| at every step and the compensation needs no
// branch (Dekker's fast two-sum error term; the same result as KSum there).
template <class R> struct PosAcc;
template <> struct PosAcc<float> {
    float s, c;
    __device__ __forceinline__ explicit PosAcc(double v0) : s((float)v0), c(0.f) {}
    __device__ __forceinline__ void add(float v)
    {
        const float t = s + v;
        c += (s - t) + v;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
template <> struct Acc<double> {
    double s;
    __device__ __forceinline__ explicit Acc(double v0) : s(v0) {}
    // a separate rounding of each term (no multiply-add fused into the sum)
    __device__ __forceinline__ void add(double v) { s = __dadd_rn(s, v); }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct PosAcc<double> : Acc<double> {
    using Acc<double>::Acc;
};

// Eq. prtcpres: p = p0 (rho / rho0)^alpha - beta; an integer alpha (7 in
// the paper's cases) by repeated squaring instead of the general power.
__device__ __forceinline__ double eos_pressure(const Inst &I, double rho)
{
    const double x = rho / I.rho0;
    double xa;
    if (I.alpha_int > 0) {
        double r = 1.0, b = x;
        for (int e = I.alpha_int; e; e >>= 1) {
            if (e & 1) r *= b;
            b *= b;
        }
        xa = r;
    } else {
        xa = pow(x, I.alpha);
    }
    return I.p0 * xa - I.beta_p;
}

// Per-particle quantities the force pass reads: p/d^2 and 1/d (FP32), also
// 1/sqrt(d) (FP64), in the precision of the pair arithmetic.
template <class R>
__device__ __forceinline__ void finalize_slot(const Bufs &b, long long s, double d, double p)
{
    if constexpr (sizeof(R) == 4) {
        // FP32 records: p/d^2 beside the velocity, 1/d beside the spin
        const float df = (float)d;
        b.B32[s].w = (float)p / (df * df);
        b.C32[s].w = 1.0f / df;
    } else {
        typename Vec<R>::T4 *D = Mir<R>::D(b);
        typename Vec<R>::T4 o = D[s];
        o.x = p / (d * d);
        o.y = 1.0 / d;
        o.z = 1.0 / sqrt(d);
        D[s] = o;
    }
}

// Streaming accesses (evict-first in L2): the neighbour lists and the normals
// cache are each read or written once per pass and would otherwise push the
// particle records, which every list revisits, out of L2.
__device__ __forceinline__ int ld_stream(const int *p) { return __ldcs(p); }
__device__ __forceinline__ float4 ld_stream(const float4 *p) { return __ldcs(p); }
__device__ __forceinline__ float2 ld_stream(const float2 *p) { return __ldcs(p); }
__device__ __forceinline__ double2 ld_stream(const double2 *p) { return __ldcs(p); }
__device__ __forceinline__ double4_32a ld_stream(const double4_32a *p)
{
    const double2 a = __ldcs((const double2 *)p), b = __ldcs((const double2 *)p + 1);
    return make_double4_32a(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st_stream(float4 *p, float4 v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(float2 *p, float2 v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(double2 *p, double2 v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(double4_32a *p, double4_32a v)
{
    __stcs((double2 *)p, make_double2(v.x, v.y));
    __stcs((double2 *)p + 1, make_double2(v.z, v.w));
}

// Persistent pair kernels: each warp takes the next 32 slots from a counter
// (zeroed before the launch) until none are left, so that no SM idles in the
// tail of a partial last wave.  The result of a slot does not depend on
// which warp computes it.
__device__ __forceinline__ long long next_warp_slots(const Bufs &b)
{
    unsigned long long base = 0;
    if ((threadIdx.x & 31) == 0) base = atomicAdd(b.work, 32ull);
    return (long long)__shfl_sync(0xffffffffu, base, 0);
}

// ------------------------------------------------------------------ density
// gate: nullptr = always; else only when *gate != 0 (a build just happened)
// Visits the entries k = 0 .. n-1 of a slot's neighbour list in order,
// calling f(k, entry, record of the partner, side value of the partner).  The
// list index two entries ahead and the record (and side value, when `side`
// is given) one entry ahead are fetched before f runs on the current one, so
// the loads of the next pair overlap this pair's arithmetic.  NB_FAR entries
// are visited too (their record is fetched without the flag bit).
template <class T4, class F>
__device__ __forceinline__ void for_each_entry(const int *__restrict__ nb, long long Np, int n,
                                               const T4 *__restrict__ A, const double *__restrict__ side, F &&f)
{
    if (n <= 0) return;
    uint32_t en = (uint32_t)ld_stream(nb);
    uint32_t enn = n > 1 ? (uint32_t)ld_stream(nb + Np) : 0u;
    T4 An = A[en & ~NB_FAR];
    double Sn = side ? side[en & ~NB_FAR] : 0.0;
    for (int k = 0; k < n; ++k) {
        const uint32_t e = en;
        const T4 Aj = An;
        const double Sj = Sn;
        if (k + 1 < n) {
            en = enn;
            An = A[en & ~NB_FAR];
            if (side) Sn = side[en & ~NB_FAR];
            if (k + 2 < n) enn = (uint32_t)ld_stream(nb + (long long)(k + 2) * Np);
        }
        f(k, e, Aj, Sj);
    }
}

template <class R, bool CLOSE>
__global__ void __launch_bounds__(256) k_density(Bufs b, int any_filter, const int *gate)
{
    if (gate && *gate == 0) return;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s == 0) *b.aclose_ok = 1;   // the marks below are for these positions
    if (s >= b.N) return;
    const int gi = b.perm[s];
    const Inst &I = b.inst[b.pinst[gi]];
    const int ti = b.stype[s];
    // mark particles with a mobile neighbour inside the collision radius of
    // the artificial viscosity (a superset: the collision pass decides exactly)
    // (CLOSE: some instance of the context has the artificial viscosity)
    const bool want_close = CLOSE && I.artvis && (ti == T_FLUID || ti == T_RIGID);
    const R close_r2 = (R)(I.artvis_r2f_hi * 1.0001f);
    bool close = false;
    double d;
    if (ti == T_OUTER) {
        d = I.inv_dx3;  // outer-wall particles are not updated (Section 2.5)
    } else {
        const auto *A = Mir<R>::A(b);
        const auto Ai = A[s];
        const Geo<R> geo(I);
        const int n = b.ncnt[s];
        const long long Np = b.Npad;
        const R Wc = K<R>::Wc(I), irc = K<R>::inv_rc(I);
        PosAcc<R> acc(I.W0);
        for_each_entry(b.nbr + s, Np, n, A, nullptr, [&](int, uint32_t e, const decltype(Ai) &Aj, double) {
            if (e & NB_FAR) return;
            R rx, ry, rz, r2;
            if (!Rel<R>::get(b, I, geo, Ai, Aj, gi, (int)e, rx, ry, rz, r2)) return;
            if (CLOSE && want_close && r2 <= close_r2) {
                const int tj = mir_type(Aj);
                close |= (tj == T_FLUID || tj == T_RIGID);
            }
            // float: correctly rounded sqrt; double: r2 / sqrt via rsqrt (~1 ulp)
            const R q = (sizeof(R) == 4 ? sqrt(r2) : r2 * rsqrt_<R>(r2)) * irc;
            const R om = lt_nonneg(q, R(1)) ? R(1) - q : R(0);
            acc.add(Wc * (R(1) + R(3) * q) * om * om * om);
        });
        d = I.Cn * acc.value();
    }
    const double rho = I.mf * d;
    double p = eos_pressure(I, rho);
    if (I.clamp && p < 0.0) p = 0.0;
    b.aclose[s] = close ? 1 : 0;
    b.sd[s] = d;
    b.sp[s] = p;
    if (!any_filter) {
        b.sp2[s] = p;
        finalize_slot<R>(b, s, d, p);
    }
}

// FP64 density with each unordered pair evaluated once (Newton 3): phase 1
// sums W over the owned prefix of the list and stores each W for the partner
// (negated when the pair lies inside the collision radius of the artificial
// viscosity; 0 for pairs beyond h) in the partner's column of the pair
// buffer, which is free between force passes (a scattered store, which does
// not stall the thread); phase 2 reads its own column in entry order
// (coalesced).  The partner's r_ji = -r_ij bit for bit and the terms are
// summed in list order ([owned][not owned]) as in k_density, so the result is
// the same.
__device__ __forceinline__ void density_half_slot(const Bufs &b, long long s)
{
    if (s >= b.N) return;
    const int gi = b.perm[s];
    const Inst &I = b.inst[b.pinst[gi]];
    const int ti = b.stype[s];
    const double4_32a *A = Mir<double>::A(b);
    const double4_32a Ai = A[s];
    const Geo<double> geo(I);
    const int nf = b.nfirst[s];
    const long long Np = b.Npad;
    double *__restrict__ wb = (double *)b.resB;
    const uint16_t *__restrict__ rv = b.rev + s;
    const double close_r2 = (double)(I.artvis_r2f_hi * 1.0001f);
    const bool want_close = I.artvis != 0;
    bool close = false;
    const double irc = K<double>::inv_rc(I), Wc = K<double>::Wc(I);
    const int capown = b.capown;
    double acc = I.W0;
    for_each_entry(b.nbr + s, Np, nf, A, nullptr, [&](int k, uint32_t e, const double4_32a &Aj, double) {
        double W = 0.0;
        if (!(e & NB_FAR)) {
            double rx, ry, rz, r2;
            if (Rel<double>::get(b, I, geo, Ai, Aj, gi, (int)e, rx, ry, rz, r2)) {
                const double q = r2 * rsqrt_<double>(r2) * irc;
                const double om = lt_nonneg(q, 1.0) ? 1.0 - q : 0.0;
                W = Wc * (1.0 + 3.0 * q) * om * om * om;
                acc = __dadd_rn(acc, W);
                if (want_close && r2 <= close_r2) {
                    const int tj = mir_type(Aj);
                    const bool mob = (tj == T_FLUID || tj == T_RIGID);
                    if (mob && (ti == T_FLUID || ti == T_RIGID)) {
                        close = true;
                        W = -W;   // tells the partner
                    }
                }
            }
        }
        // into the partner's column, at the row of its entry for this pair
        const int row = __ldg(rv + (long long)k * Np);
        if (row < capown) wb[(long long)row * Np + (e & ~NB_FAR)] = W;
    });
    b.sd[s] = acc;   // partial; completed by k_density_gather
    b.aclose[s] = close ? 1 : 0;
}

__global__ void __launch_bounds__(256) k_density_half(Bufs b, const int *gate)
{
    if (gate && *gate == 0) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) *b.aclose_ok = 1;
    for (long long base = next_warp_slots(b); base < b.N; base = next_warp_slots(b))
        density_half_slot(b, base + (threadIdx.x & 31));
}

__global__ void __launch_bounds__(256) k_density_gather(Bufs b, int any_filter, const int *gate)
{
    if (gate && *gate == 0) return;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.N) return;
    const int gi = b.perm[s];
    const Inst &I = b.inst[b.pinst[gi]];
    const int ti = b.stype[s];
    double d;
    if (ti == T_OUTER) {
        d = I.inv_dx3;  // outer-wall particles are not updated (Section 2.5)
    } else {
        const double *__restrict__ wb = (const double *)b.resB;
        const int n = b.ncnt[s], nf = b.nfirst[s];
        const long long Np = b.Npad;
        // the owners wrote W of this particle's non-owned entries into its
        // own column (row k - nf; more rows than capown only after a list
        // error, flagged)
        const int nend = min(n, nf + b.capown);
        double acc = b.sd[s];
        bool close = b.aclose[s] != 0;
        constexpr int G = 4;
        for (int k0 = nf; k0 < nend; k0 += G) {
            double w[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int k = k0 + g;
                w[g] = 0.0;
                if (k < nend) {
                    const uint32_t e = (uint32_t)__ldg(b.nbr + (long long)k * Np + s);
                    if (!(e & NB_FAR)) w[g] = wb[(long long)(k - nf) * Np + s];
                }
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (w[g] < 0.0) close = true;
                acc = __dadd_rn(acc, fabs(w[g]));
            }
        }
        d = I.Cn * acc;
        b.aclose[s] = (close && (ti == T_FLUID || ti == T_RIGID)) ? 1 : 0;
    }
    const double rho = I.mf * d;
    double p = eos_pressure(I, rho);
    if (I.clamp && p < 0.0) p = 0.0;
    b.sd[s] = d;
    b.sp[s] = p;
    if (!any_filter) {
        b.sp2[s] = p;
        finalize_slot<double>(b, s, d, p);
    }
}

// ------------------------------------------------------ density reinitialisation
// Shepard reinitialisation of the summation density (after Colagrossi and
// Landrini; the text under Algorithm 1): d~_i = (W(0) + sum_j W_ij) /
// (W(0)/d_i + sum_j W_ij/d_j) over the density neighbours, outer walls keep
// theirs; the pressure follows from Eq. prtcpres.  The new densities go to
// sdr (the neighbours' old values are still read) and k_reinit_copy moves
// them back.
template <class R>
__global__ void __launch_bounds__(256) k_reinit(Bufs b, int any_filter, const int *gate)
{
    if (gate && *gate == 0) return;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.N) return;
    const int gi = b.perm[s];
    const Inst &I = b.inst[b.pinst[gi]];
    const double di = b.sd[s];
    double d = di;
    if (I.reinit && b.stype[s] != T_OUTER) {
        const auto *A = Mir<R>::A(b);
        const auto Ai = A[s];
        const Geo<R> geo(I);
        const int n = b.ncnt[s];
        const long long Np = b.Npad;
        const R Wc = K<R>::Wc(I), irc = K<R>::inv_rc(I);
        Acc<R> num(I.W0), den(I.W0 / di);
        for_each_entry(b.nbr + s, Np, n, A, b.sd, [&](int, uint32_t e, const decltype(Ai) &Aj, double dj) {
            if (e & NB_FAR) return;
            R rx, ry, rz, r2;
            if (!Rel<R>::get(b, I, geo, Ai, Aj, gi, (int)e, rx, ry, rz, r2)) return;
            const R q = sqrt(r2) * irc;
            const R om = lt_nonneg(q, R(1)) ? R(1) - q : R(0);
            const R W = Wc * (R(1) + R(3) * q) * om * om * om;
            num.add(W);
            den.add(W / (R)dj);
        });
        d = num.value() / den.value();
    }
    const double rho = I.mf * d;
    double p = eos_pressure(I, rho);
    if (I.clamp && p < 0.0) p = 0.0;
    b.sdr[s] = d;
    if (I.reinit) b.sp[s] = p;
    if (!any_filter) {
        b.sp2[s] = b.sp[s];
        finalize_slot<R>(b, s, d, b.sp[s]);
    }
}

__global__ void k_reinit_copy(Bufs b, const int *gate)
{
    if (gate && *gate == 0) return;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < b.N) b.sd[s] = b.sdr[s];
}

// ------------------------------------------------------------ pressure filter
template <class R>
__global__ void __launch_bounds__(256) k_filter(Bufs b, const int *gate)
{
    if (gate && *gate == 0) return;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.N) return;
    const int gi = b.perm[s];
    const Inst &I = b.inst[b.pinst[gi]];
    const double pi = b.sp[s];
    double pf = pi;
    if (I.filter && b.stype[s] != T_OUTER) {
        const auto *A = Mir<R>::A(b);
        const auto Ai = A[s];
        const Geo<R> geo(I);
        const int n = b.ncnt[s];
        const long long Np = b.Npad;
        const R Wc = K<R>::Wc(I), irc = K<R>::inv_rc(I);
        Acc<R> num(pi * I.W0), den(I.W0);
        for_each_entry(b.nbr + s, Np, n, A, b.sp, [&](int, uint32_t e, const decltype(Ai) &Aj, double pj) {
            if (e & NB_FAR) return;
            R rx, ry, rz, r2;
            if (!Rel<R>::get(b, I, geo, Ai, Aj, gi, (int)e, rx, ry, rz, r2)) return;
            const R q = sqrt(r2) * irc;
            const R om = lt_nonneg(q, R(1)) ? R(1) - q : R(0);
            const R W = Wc * (R(1) + R(3) * q) * om * om * om;
            num.add((R)pj * W);
            den.add(W);
        });
        pf = num.value() / den.value();
    }
    b.sp2[s] = pf;
    finalize_slot<R>(b, s, b.sd[s], pf);
}

// ---------------------------------------------------------------- drag (A5)
// r = x_i - x_j with the minimum image; returns the oracle's r^2 (no FMA).
__device__ __forceinline__ double exact_disp(const double *xi, const double *xj, const Inst &I, double r[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double t = __dsub_rn(xi[a], xj[a]);
        if (I.periodic[a]) {
            const double hL = 0.5 * I.box[a];
            if (t > hL) t = __dsub_rn(t, I.box[a]);
            else if (t < -hL) t = __dadd_rn(t, I.box[a]);
        }
        r[a] = t;
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(r[0], r[0]), __dmul_rn(r[1], r[1])), __dmul_rn(r[2], r[2]));
}

// The sphere kernels run one warp per rigid particle, RB / 32 particles per
// block: the lanes stride over its neighbour list and the partial sums are
// reduced by a fixed butterfly of shuffles, so the result does not depend on
// scheduling.
constexpr int RB = 128;
constexpr int RPB = RB / 32;   // rigid particles per block

template <int K>
__device__ __forceinline__ void warp_sum_all(double (&v)[K])
{
#pragma unroll
    for (int a = 0; a < K; ++a) v[a] = warp_sum(v[a]);
}

// Per rigid particle s (one warp each, lanes striding over its neighbour
// list, order-fixed reduction): the rigid volume within h, sum W and
// sum W v over fluid neighbours (Eq. fvfdef, Section 2.4); k_drag_law then forms
// eps_s (s included), v_f = sum W v / sum W and the drag along (v_f - v_s)
// with the Ergun (eps <= 0.8) or Wen-Yu (eps > 0.8) coefficient in the closed
// form that stays finite at eps -> 1 and |v_f - v_s| -> 0.
template <class R>
__global__ void __launch_bounds__(RB) k_drag(Bufs b)
{
    const int r = blockIdx.x * RPB + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r >= b.nrigid) return;   // the whole warp
    const int g = b.rigid_gid[r];
    const long long s = b.slot_of[g];
    const Inst &I = b.inst[b.pinst[g]];
    double Vsum = 0.0, S = 0.0, U0 = 0.0, U1 = 0.0, U2 = 0.0;
    const int n = b.ncnt[s];
    // the kernel-weighted fluid sums in precision R on the mirrors (the
    // exact r < h decision of Rel), per lane in R; the volumes in FP64
    using T4 = typename Vec<R>::T4;
    const Geo<R> geo(I);
    const T4 *__restrict__ A = Mir<R>::A(b);
    const T4 *__restrict__ Bm = Mir<R>::B(b);
    const T4 Ai = A[s];
    const R Wc = K<R>::Wc(I), irc = K<R>::inv_rc(I);
    R Sr = 0, u0 = 0, u1 = 0, u2 = 0;
    for (int k = lane; k < n; k += 32) {
        const uint32_t e = (uint32_t)b.nbr[(long long)k * b.Npad + s];
        if (e & NB_FAR) continue;
        const int j = (int)e;
        const T4 Aj = A[j];
        const int tj = mir_type(Aj);
        if (tj != T_RIGID && tj != T_FLUID) continue;
        R rx, ry, rz, r2;
        if (!Rel<R>::get(b, I, geo, Ai, Aj, g, j, rx, ry, rz, r2)) continue;
        if (tj == T_RIGID) {
            const double Rj = b.R[b.perm[j]];
            Vsum += 4.0 / 3.0 * PI * Rj * Rj * Rj;
        } else {
            const R q = sqrt(r2) * irc, om = R(1) - q;
            const R W = Wc * (R(1) + R(3) * q) * om * om * om;
            const T4 Bj = Bm[j];
            Sr += W;
            u0 += W * Bj.x;
            u1 += W * Bj.y;
            u2 += W * Bj.z;
        }
    }
    S = Sr; U0 = u0; U1 = u1; U2 = u2;
    double sums[5] = { Vsum, S, U0, U1, U2 };
    warp_sum_all(sums);
    if (lane == 0)
        for (int a = 0; a < 5; ++a) b.dsum[5 * r + a] = sums[a];
}

// The drag law of each rigid particle from its sums (one thread each, so the
// FP64 power functions of many particles run side by side).
__global__ void k_drag_law(Bufs b)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= b.nrigid) return;
    const int g = b.rigid_gid[r];
    const long long s = b.slot_of[g];
    const Inst &I = b.inst[b.pinst[g]];
    const double Ri = b.R[g];
    const double *sums = b.dsum + 5 * r;
    const double Vsum = sums[0] + 4.0 / 3.0 * PI * Ri * Ri * Ri;
    const double S = sums[1];
    const double U[3] = { sums[2], sums[3], sums[4] };
    double eps = fabs(I.Vf - Vsum) / I.Vf;
    eps = fmin(fmax(eps, I.eps_min), 1.0);
    double F[3] = { 0.0, 0.0, 0.0 };
    if (S > 0.0) {
        double dv[3];
        for (int a = 0; a < 3; ++a) dv[a] = U[a] / S - b.v[3 * g + a];
        const double mag = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        const double d = 2.0 * Ri, Vs = 4.0 / 3.0 * PI * Ri * Ri * Ri;
        double coef;
        if (eps <= 0.8) {
            coef = 150.0 * I.eta * (1.0 - eps) / (eps * d * d) + 1.75 * I.rho0 * mag / d;
        } else {
            const double Re = I.rho0 * d * eps * mag / I.eta;
            const double cdre = (Re <= 1000.0) ? 24.0 * (1.0 + 0.15 * pow(Re, 0.687)) : 0.44 * Re;
            coef = 0.75 * cdre * I.eta * pow(eps, -2.65) / (d * d);
        }
        for (int a = 0; a < 3; ++a) F[a] = coef * Vs * dv[a];
        b.rxn[s] = make_double4_32a(F[0] / S, F[1] / S, F[2] / S, 0.0);
        b.rxn32[s] = make_float4((float)(F[0] / S), (float)(F[1] / S), (float)(F[2] / S), 0.f);
    } else {
        b.rxn[s] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        b.rxn32[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    b.eps[r] = eps;
    b.fdg[3 * r] = F[0];
    b.fdg[3 * r + 1] = F[1];
    b.fdg[3 * r + 2] = F[2];
}

// External acceleration (Eq. govern, F^EXT): uniform g plus the
// reverse-Poiseuille forcing, + on the lower half of split_axis, - above.
__device__ __forceinline__ void ext_accel(const Inst &I, const double *x, double a[3])
{
    a[0] = I.g[0];
    a[1] = I.g[1];
    a[2] = I.g[2];
    if (I.body_amp != 0.0) {
        const double rel = x[I.split_axis] - I.origin[I.split_axis];
        a[I.body_axis] += (rel < 0.5 * I.box[I.split_axis]) ? I.body_amp : -I.body_amp;
    }
}

// -------------------------------------------------------- fluid force pass
// Constants of the SDPD pair force in precision R, held in registers.
// Products of instance constants are folded once per thread:
//   A1 = -cd Ca, A2 = cd (Ca + 2 Cb) / 3, A3 = -cr Ca / 2 (Eqs. FijD, FijR with
//   gamma_a = Ca F/(d_i d_j), gamma_b = Cb F/(d_i d_j)); T1 = ct Ka / sqrt(dt),
//   T3 = ct (Kb - Ka) / (3 sqrt(dt)) (Eq. FijT with sigma = K sqrt(F)/sqrt(d_i d_j)).
template <class R> struct PairK {
    R irc, Fc, Wc, cc, A1, A2, A3, T1, T3, lev;
    bool noise;
    uint32_t step, key0, key1;
    __device__ __forceinline__ PairK(const Inst &I, uint32_t st)
        : irc(K<R>::inv_rc(I)), Fc(K<R>::Fc(I)), Wc(K<R>::Wc(I)), cc(K<R>::cc(I)),
          A1(-K<R>::cd(I) * K<R>::Ca(I)),
          A2(K<R>::cd(I) * (K<R>::Ca(I) + R(2) * K<R>::Cb(I)) * R(1.0 / 3.0)),
          A3(R(-0.5) * K<R>::cr(I) * K<R>::Ca(I)),
          T1(K<R>::ct(I) * K<R>::isdt(I) * K<R>::Ka(I)),
          T3(K<R>::ct(I) * K<R>::isdt(I) * (K<R>::Kb(I) - K<R>::Ka(I)) * R(1.0 / 3.0)),
          lev(K<R>::lever(I)), noise(I.noise != 0), step(st), key0(I.key0), key1(I.key1) {}
};


// Correctly rounded operations in precision R that the compiler may not
// contract or reorder.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// Kernel weight W(r) = Wc (1 + 3q)(1 - q)^3 of a pair for the drag reaction
// (Eq. F_fpi_DG_reac), every rounding explicit.
template <class R>
__device__ __forceinline__ R drag_weight(const PairK<R> &P, R q, R om)
{
    return mul_rn(mul_rn(mul_rn(mul_rn(P.Wc, fma_rn(R(3), q, R(1))), om), om), om);
}

template <class R> struct Z6 {
    R z0, z1, z2, z3, z4, z5;
};

// f = o + ce e and h = e x o of a pair in a fixed operation order, so that
// the partner of the split path, which rebuilds them from {o, ce} and its
// own (negated, bitwise equal) e, gets the owner's values exactly.
__device__ __forceinline__ void pair_fh(float ox, float oy, float oz, float ce, float ex, float ey, float ez,
                                        float &gx, float &gy, float &gz, float &hx, float &hy, float &hz)
{
    gx = __fmaf_rn(ce, ex, ox);
    gy = __fmaf_rn(ce, ey, oy);
    gz = __fmaf_rn(ce, ez, oz);
    hx = __fmaf_rn(ey, oz, -__fmul_rn(ez, oy));
    hy = __fmaf_rn(ez, ox, -__fmul_rn(ex, oz));
    hz = __fmaf_rn(ex, oy, -__fmul_rn(ey, ox));
}
__device__ __forceinline__ void pair_fh(double ox, double oy, double oz, double ce, double ex, double ey, double ez,
                                        double &gx, double &gy, double &gz, double &hx, double &hy, double &hz)
{
    gx = fma(ce, ex, ox);
    gy = fma(ce, ey, oy);
    gz = fma(ce, ez, oz);
    hx = fma(ey, oz, -__dmul_rn(ez, oy));
    hy = fma(ez, ox, -__dmul_rn(ex, oz));
    hz = fma(ex, oy, -__dmul_rn(ey, ox));
}

// SDPD force on i from j (Eqs. FijC, FijD, FijR, FijT) for a pair already
// known to lie within h, written as
//   f = o + ce * e,   o = the part not along e_ij (v_ij, rotational, random),
// so the torque (-l e) x f = -l e x o needs only o.  with_rt: rotational and
// random parts (not for pairs with a rigid particle, Section 2.4).  zmode:
// 0 draw the six normals into z, 1 use z as given.  Also returns e, q, 1 - q.
template <class R, class T4>
__device__ __forceinline__ void sdpd_pair(const PairK<R> &P, R rx, R ry, R rz, R r2, const T4 &Bi,
                                          const T4 &Ci, const T4 &Di, const T4 &Bj, const T4 &Cj,
                                          const T4 &Dj, bool with_rt, int zmode, Z6<R> &z, R &ox,
                                          R &oy, R &oz, R &ce, R &ex, R &ey, R &ez, R &q, R &om)
{
    const R is2 = R(0.70710678118654752440);
    const R ir = rsqrt_<R>(r2);
    q = r2 * ir * P.irc;
    om = lt_nonneg(q, R(1)) ? R(1) - q : R(0);
    const R Fk = P.Fc * om * om;
    ex = rx * ir; ey = ry * ir; ez = rz * ir;
    const R vx = Bi.x - Bj.x, vy = Bi.y - Bj.y, vz = Bi.z - Bj.z;
    const R ev = ex * vx + ey * vy + ez * vz;
    const R gf = Fk * mir_invd(Ci, Di) * mir_invd(Cj, Dj);
    const R c1 = P.A1 * gf;
    // Eq. FijC (central) + the central part of Eq. FijD
    ce = P.cc * (mir_pd2(Bi, Di) + mir_pd2(Bj, Dj)) * Fk * (r2 * ir) - P.A2 * gf * ev;
    ox = c1 * vx; oy = c1 * vy; oz = c1 * vz;
    if (!with_rt) return;
    // Eq. FijR
    const R wx = Ci.x + Cj.x, wy = Ci.y + Cj.y, wz = Ci.z + Cj.z;
    const R c3 = P.A3 * gf;
    ox += c3 * (ry * wz - rz * wy);
    oy += c3 * (rz * wx - rx * wz);
    oz += c3 * (rx * wy - ry * wx);
    // Eq. FijT: (sa S + (sb - sa) tr(S)/3 1) . e / sqrt(dt).  Every operation
    // on the normals is spelled out (no contraction left to the compiler), so
    // normals drawn here and normals read back from the cache give the same
    // force bits.
    if (P.noise) {
        if (zmode == 0)
            pair_normals<R>(mir_gid(Di), mir_gid(Dj), P.step, P.key0, P.key1, z.z0, z.z1, z.z2, z.z3,
                            z.z4, z.z5);
        const R rs = mir_rs(om, Ci, Di, Cj, Dj);
        const R sa = P.T1 * rs;
        const R sxy = mul_rn(z.z3, is2), sxz = mul_rn(z.z4, is2), syz = mul_rn(z.z5, is2);
        ce = fma_rn(P.T3 * rs, add_rn(add_rn(z.z0, z.z1), z.z2), ce);
        ox = fma_rn(sa, fma_rn(sxz, ez, fma_rn(sxy, ey, mul_rn(z.z0, ex))), ox);
        oy = fma_rn(sa, fma_rn(syz, ez, fma_rn(z.z1, ey, mul_rn(sxy, ex))), oy);
        oz = fma_rn(sa, fma_rn(z.z2, ez, fma_rn(syz, ey, mul_rn(sxz, ex))), oz);
    }
}

template <class R>
__device__ __forceinline__ void write_fluid_force(const Bufs &b, const Inst &I, int gi, R fx, R fy,
                                                  R fz, R tx, R ty, R tz, R lev)
{
    double a[3];
    const double xg[3] = { b.x[3 * gi], b.x[3 * gi + 1], b.x[3 * gi + 2] };
    ext_accel(I, xg, a);
    const double m = b.m[gi];
    b.F[3 * gi] = (double)fx + m * a[0];
    b.F[3 * gi + 1] = (double)fy + m * a[1];
    b.F[3 * gi + 2] = (double)fz + m * a[2];
    b.T[3 * gi] = -(double)(lev * tx);
    b.T[3 * gi + 1] = -(double)(lev * ty);
    b.T[3 * gi + 2] = -(double)(lev * tz);
}

// F^DG_s / S_s of rigid slot j in precision R (Eq. F_fpi_DG_reac).
__device__ __forceinline__ void rxn_of(const Bufs &b, int j, float &x, float &y, float &z)
{
    const float4 r = b.rxn32[j];
    x = r.x; y = r.y; z = r.z;
}
__device__ __forceinline__ void rxn_of(const Bufs &b, int j, double &x, double &y, double &z)
{
    const double4_32a r = b.rxn[j];
    x = r.x; y = r.y; z = r.z;
}

// Fluid particle i and a rigid neighbour j (Section 2.4): Eqs. FijC and FijD
// on i (no rotational or random part) and the drag reaction Eq.
// F_fpi_DG_reac, added to i's sums; nothing beyond h.
template <class R, class T4>
__device__ __forceinline__ void fluid_rigid_pair(const Bufs &b, const Inst &I, const Geo<R> &geo,
                                                 const PairK<R> &P, int gi, const T4 &Ai, const T4 &Bi,
                                                 const T4 &Ci, const T4 &Di, int j, const T4 &Aj,
                                                 const T4 &Bj, const T4 &Cj, const T4 &Dj, R &fx, R &fy,
                                                 R &fz, R &tx, R &ty, R &tz)
{
    R rx, ry, rz, r2;
    if (!Rel<R>::get(b, I, geo, Ai, Aj, gi, j, rx, ry, rz, r2)) return;
    R ox, oy, oz, ce, ex, ey, ez, q, om;
    Z6<R> z;
    sdpd_pair<R>(P, rx, ry, rz, r2, Bi, Ci, Di, Bj, Cj, Dj, false, 0, z, ox, oy, oz, ce, ex, ey, ez, q, om);
    R rcx, rcy, rcz;
    rxn_of(b, j, rcx, rcy, rcz);
    const R W = P.Wc * (R(1) + R(3) * q) * om * om * om;
    fx += ox + ce * ex - rcx * W;
    fy += oy + ce * ey - rcy * W;
    fz += oz + ce * ez - rcz * W;
    tx += ey * oz - ez * oy;
    ty += ez * ox - ex * oz;
    tz += ex * oy - ey * ox;
}

// The same, called out of line where rigid neighbours are rare and the
// caller's registers matter (the gather), loading the records itself.
template <class R>
__device__ __noinline__ void fluid_rigid_pair_call(const Bufs &b, long long s, int gi, int j, R *f)
{
    using T4 = typename Vec<R>::T4;
    const Inst &I = b.inst[b.pinst[gi]];
    const Geo<R> geo(I);
    const PairK<R> P(I, (uint32_t)(*b.step));
    const T4 *__restrict__ A = Mir<R>::A(b);
    const T4 *__restrict__ Bm = Mir<R>::B(b);
    const T4 *__restrict__ Cm = Mir<R>::C(b);
    const T4 *__restrict__ Dm = Mir<R>::D(b);
    fluid_rigid_pair<R>(b, I, geo, P, gi, A[s], Bm[s], Cm[s], Dm[s], j, A[j], Bm[j], Cm[j], Dm[j], f[0], f[1],
                        f[2], f[3], f[4], f[5]);
}

// Direct (owner-computes-all) force pass over the neighbour list of fluid
// particle i.  The index two entries ahead and the records of the next
// neighbour are fetched before the current pair is evaluated.  With the
// cache on, the first evaluation of a step (FILL) stores the six normals of
// every entry in its own column (a NaN marker for an entry beyond h); the
// second (REUSE, when the list has not been rebuilt in between) reads them
// back, fetched one entry ahead like the records, instead of drawing them
// again (same counter, so the same bits).
template <class R, bool REUSE>
__device__ __forceinline__ void force_fluid_slot(const Bufs &b, long long s, uint32_t step, bool fill)
{
    // FP32, normals from the cache: a partner's D record (its gid) only for a
    // pair whose normals must be drawn after all (rare), loaded then
    constexpr bool LAZY_D = REUSE && sizeof(R) == 4;
    using T4 = typename Vec<R>::T4;
    using T2 = typename Vec2<R>::T2;
    if (s >= b.N) return;
    if (b.stype[s] != T_FLUID) return;
    const int gi = b.perm[s];
    const Inst &I = b.inst[b.pinst[gi]];
    const Geo<R> geo(I);
    const PairK<R> P(I, step);
    fill = fill && P.noise;
    const T4 *__restrict__ A = Mir<R>::A(b);
    const T4 *__restrict__ Bm = Mir<R>::B(b);
    const T4 *__restrict__ Cm = Mir<R>::C(b);
    const T4 *__restrict__ Dm = Mir<R>::D(b);
    T4 *__restrict__ zA = (T4 *)b.zdA;
    T2 *__restrict__ zB = (T2 *)b.zdB;
    const int *__restrict__ nb = b.nbr + s;
    const T4 Ai = A[s], Bi = Bm[s], Ci = Cm[s], Di = Dm[s];
    R fx = 0, fy = 0, fz = 0, tx = 0, ty = 0, tz = 0;
    const int n = b.ncnt[s];
    const long long Np = b.Npad;
    int jn = n > 0 ? ld_stream(nb) : 0;
    int jnn = n > 1 ? ld_stream(nb + Np) : 0;
    T4 An = A[jn], Bn = Bm[jn], Cn = Cm[jn], Dn = Di;
    if constexpr (!LAZY_D) Dn = Dm[jn];
    T4 zan;
    T2 zbn;
    if (REUSE && P.noise && n > 0) { zan = ld_stream(zA + s); zbn = ld_stream(zB + s); }
    for (int k = 0; k < n; ++k) {
        const int j = jn;
        const T4 Aj = An, Bj = Bn, Cj = Cn;
        T4 Dj = Dn;
        T4 za;
        T2 zb;
        if (REUSE) { za = zan; zb = zbn; }
        if (k + 1 < n) {
            jn = jnn;
            An = A[jn]; Bn = Bm[jn]; Cn = Cm[jn];
            if constexpr (!LAZY_D) Dn = Dm[jn];
            if (REUSE && P.noise) {
                zan = ld_stream(zA + (long long)(k + 1) * Np + s);
                zbn = ld_stream(zB + (long long)(k + 1) * Np + s);
            }
            if (k + 2 < n) jnn = ld_stream(nb + (long long)(k + 2) * Np);
        }
        const bool rig = mir_type(Aj) == T_RIGID;
        const long long at = (long long)k * Np + s;
        R rx, ry, rz, r2;
        if (!Rel<R>::get(b, I, geo, Ai, Aj, gi, j, rx, ry, rz, r2)) {
            if (!REUSE && fill && !rig) {
                T4 nm;
                nm.x = R(NAN); nm.y = R(0); nm.z = R(0); nm.w = R(0);
                st_stream(zA + at, nm);
            }
            continue;
        }
        R ox, oy, oz, ce, ex, ey, ez, q, om;
        Z6<R> z;
        int zmode = 0;
        // an entry beyond h in the first evaluation carries the NaN marker
        if (REUSE && P.noise && !rig && !isnan(za.x)) {
            z.z0 = za.x; z.z1 = za.y; z.z2 = za.z; z.z3 = za.w; z.z4 = zb.x; z.z5 = zb.y;
            zmode = 1;
        }
        if constexpr (LAZY_D) {
            if (zmode == 0 && P.noise && !rig) Dj = Dm[j];
        }
        sdpd_pair<R>(P, rx, ry, rz, r2, Bi, Ci, Di, Bj, Cj, Dj, !rig, zmode, z, ox, oy, oz, ce, ex, ey, ez,
                     q, om);
        if (!REUSE && fill && !rig) {
            T4 zw;
            zw.x = z.z0; zw.y = z.z1; zw.z = z.z2; zw.w = z.z3;
            T2 zv;
            zv.x = z.z4; zv.y = z.z5;
            st_stream(zA + at, zw);
            st_stream(zB + at, zv);
        }
        // every accumulation step rounded explicitly (the pair-stream pass
        // adds the same terms in the same order and must match bit for bit)
        R gx, gy, gz, hx, hy, hz;
        pair_fh(ox, oy, oz, ce, ex, ey, ez, gx, gy, gz, hx, hy, hz);
        if (rig) {
            // Eq. F_fpi_DG_reac: -F^DG_s W_sj / S_s
            R rcx, rcy, rcz;
            rxn_of(b, j, rcx, rcy, rcz);
            const R W = drag_weight(P, q, om);
            fx = sub_rn(fx, mul_rn(rcx, W));
            fy = sub_rn(fy, mul_rn(rcy, W));
            fz = sub_rn(fz, mul_rn(rcz, W));
        }
        fx = add_rn(fx, gx);
        fy = add_rn(fy, gy);
        fz = add_rn(fz, gz);
        tx = add_rn(tx, hx);
        ty = add_rn(ty, hy);
        tz = add_rn(tz, hz);
    }
    write_fluid_force<R>(b, I, gi, fx, fy, fz, tx, ty, tz, P.lev);
}

// 16-byte asynchronous copy global -> shared, cached in L1 (PTX cp.async,
// sm_80 and later; measured faster here than the L2-only form), and its
// commit / wait
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Shared-memory ring of the async variant: per thread DEPTH stages of the
// partner's B, C, D records, thread-minor (rec[stage][record][thread]) so a
// warp's 16-byte accesses fall on consecutive banks.
constexpr int LEAN_BLOCK = 128;
template <int DEPTH> struct LeanRing {
    float4 rec[DEPTH][3][LEAN_BLOCK];
};

// DEPTH > 0: the partner's B, C, D records through the async ring (above)
template <class R, bool REUSE, int DEPTH = 0>
__device__ __forceinline__ void force_fluid_slot_lean(const Bufs &b, long long s, uint32_t step, bool fill,
                                                      LeanRing<DEPTH ? DEPTH : 1> *ring = nullptr)
{
    constexpr bool ASYNC = DEPTH > 0;
    // FP32, normals from the cache: a partner's D record (its gid) is needed
    // only for a pair whose normals must be drawn after all (rare), so it is
    // loaded then
    constexpr bool LAZY_D = REUSE && sizeof(R) == 4;
    using T4 = typename Vec<R>::T4;
    using T2 = typename Vec2<R>::T2;
    if (s >= b.N) return;
    if (b.stype[s] != T_FLUID) return;
    const int gi = b.perm[s];
    const Inst &I = b.inst[b.pinst[gi]];
    const Geo<R> geo(I);
    const PairK<R> P(I, step);
    fill = fill && P.noise;
    const T4 *__restrict__ A = Mir<R>::A(b);
    const T4 *__restrict__ Bm = Mir<R>::B(b);
    const T4 *__restrict__ Cm = Mir<R>::C(b);
    const T4 *__restrict__ Dm = Mir<R>::D(b);
    T4 *__restrict__ zA = (T4 *)b.zdA;
    T2 *__restrict__ zB = (T2 *)b.zdB;
    const int *__restrict__ nb = b.nbr + s;
    const T4 Ai = A[s], Bi = Bm[s], Ci = Cm[s], Di = Dm[s];
    R fx = 0, fy = 0, fz = 0, tx = 0, ty = 0, tz = 0;
    const int n = b.ncnt[s];
    const long long Np = b.Npad;
    int jn = n > 0 ? ld_stream(nb) : 0;
    int jnn = n > 1 ? ld_stream(nb + Np) : 0;
    T4 An = A[jn];
    T4 zan;
    T2 zbn;
    if (REUSE && P.noise && n > 0) { zan = ld_stream(zA + s); zbn = ld_stream(zB + s); }
    const int lt = threadIdx.x;
    // async ring: the records of entry k + DEPTH - 1 go in flight while entry
    // k is evaluated; one commit group per entry keeps the wait count fixed
    auto request = [&](int kk, int jj) {
        if constexpr (ASYNC) {
            if (kk < n) {
                const int st = kk % DEPTH;
                cp_async16(&ring->rec[st][0][lt], Bm + jj);
                cp_async16(&ring->rec[st][1][lt], Cm + jj);
                cp_async16(&ring->rec[st][2][lt], Dm + jj);
            }
            cp_async_commit();
        }
    };
    // entries 0 .. DEPTH-2 requested before the loop (0 and 1 are jn, jnn);
    // jq: the list entry DEPTH - 1 ahead, the next to request
    int jq = 0;
    if constexpr (ASYNC) {
        request(0, jn);
        if constexpr (DEPTH > 2) request(1, jnn);
#pragma unroll
        for (int d = 2; d < DEPTH; ++d) {
            const int e = d < n ? ld_stream(nb + (long long)d * Np) : 0;
            if (d + 1 < DEPTH) request(d, e);
            else jq = e;
        }
    }
    for (int k = 0; k < n; ++k) {
        if constexpr (ASYNC) {
            // the partner DEPTH - 1 entries ahead, whether or not it is within
            // h, into the stage of entry k - 1, whose copies are complete
            // first (an entry beyond h is never waited for at its use)
            cp_async_wait<DEPTH - 1>();
            if constexpr (DEPTH == 2) {
                request(k + 1, jnn);
            } else {
                request(k + DEPTH - 1, jq);
                if (k + DEPTH < n) jq = ld_stream(nb + (long long)(k + DEPTH) * Np);
            }
        }
        const int j = jn;
        const T4 Aj = An;
        T4 za;
        T2 zb;
        if (REUSE) { za = zan; zb = zbn; }
        if (k + 1 < n) {
            jn = jnn;
            An = A[jn];
            if (REUSE && P.noise) {
                zan = ld_stream(zA + (long long)(k + 1) * Np + s);
                zbn = ld_stream(zB + (long long)(k + 1) * Np + s);
            }
            if (k + 2 < n) jnn = ld_stream(nb + (long long)(k + 2) * Np);
        }
        const bool rig = mir_type(Aj) == T_RIGID;
        const long long at = (long long)k * Np + s;
        R rx, ry, rz, r2;
        if (!Rel<R>::get(b, I, geo, Ai, Aj, gi, j, rx, ry, rz, r2)) {
            if (!REUSE && fill && !rig) {
                T4 nm;
                nm.x = R(NAN); nm.y = R(0); nm.z = R(0); nm.w = R(0);
                st_stream(zA + at, nm);
            }
            continue;
        }
        T4 Bj, Cj, Dj = Di;
        if constexpr (ASYNC) {
            cp_async_wait<DEPTH - 1>();   // this entry's group is complete
            const int st = k % DEPTH;
            Bj = ring->rec[st][0][lt];
            Cj = ring->rec[st][1][lt];
            Dj = ring->rec[st][2][lt];
        } else {
            Bj = Bm[j];
            Cj = Cm[j];
            if constexpr (!LAZY_D) Dj = Dm[j];
        }
        R ox, oy, oz, ce, ex, ey, ez, q, om;
        Z6<R> z;
        int zmode = 0;
        // an entry beyond h in the first evaluation carries the NaN marker
        if (REUSE && P.noise && !rig && !isnan(za.x)) {
            z.z0 = za.x; z.z1 = za.y; z.z2 = za.z; z.z3 = za.w; z.z4 = zb.x; z.z5 = zb.y;
            zmode = 1;
        }
        if constexpr (LAZY_D) {
            if (zmode == 0 && P.noise && !rig) Dj = Dm[j];
        }
        sdpd_pair<R>(P, rx, ry, rz, r2, Bi, Ci, Di, Bj, Cj, Dj, !rig, zmode, z, ox, oy, oz, ce, ex, ey, ez,
                     q, om);
        if (!REUSE && fill && !rig) {
            T4 zw;
            zw.x = z.z0; zw.y = z.z1; zw.z = z.z2; zw.w = z.z3;
            T2 zv;
            zv.x = z.z4; zv.y = z.z5;
            st_stream(zA + at, zw);
            st_stream(zB + at, zv);
        }
        // every accumulation step rounded explicitly (the pair-stream pass
        // adds the same terms in the same order and must match bit for bit)
        R gx, gy, gz, hx, hy, hz;
        pair_fh(ox, oy, oz, ce, ex, ey, ez, gx, gy, gz, hx, hy, hz);
        if (rig) {
            // Eq. F_fpi_DG_reac: -F^DG_s W_sj / S_s
            R rcx, rcy, rcz;
            rxn_of(b, j, rcx, rcy, rcz);
            const R W = drag_weight(P, q, om);
            fx = sub_rn(fx, mul_rn(rcx, W));
            fy = sub_rn(fy, mul_rn(rcy, W));
            fz = sub_rn(fz, mul_rn(rcz, W));
        }
        fx = add_rn(fx, gx);
        fy = add_rn(fy, gy);
        fz = add_rn(fz, gz);
        tx = add_rn(tx, hx);
        ty = add_rn(ty, hy);
        tz = add_rn(tz, hz);
    }
    if constexpr (ASYNC) cp_async_wait<0>();   // nothing left in flight into the ring
    write_fluid_force<R>(b, I, gi, fx, fy, fz, tx, ty, tz, P.lev);
}

// The direct pass with only the list index and the partner's position
// fetched ahead (its other records are loaded after the r < h decision):
// fewer registers, so more warps per SM hide the loads instead (force mode
// 5; the same terms in the same order, so the same bits as force_fluid_slot).
// ONLY: 0 every path; 1 only the second evaluation that reads the cached
// normals (returns at once otherwise); 2 only the paths that draw them
template <class R, int MINB, int DEPTH = 0, int ONLY = 0>
__global__ void __launch_bounds__(LEAN_BLOCK, MINB) k_force_fluid_lean(Bufs b, int velver)
{
    LeanRing<DEPTH ? DEPTH : 1> *ring = nullptr;
    if constexpr (DEPTH > 0) {
        __shared__ LeanRing<DEPTH ? DEPTH : 1> ring_s;
        ring = &ring_s;
    }
    const uint32_t step = (uint32_t)(*b.step);
    const bool fill = b.use_cache && velver == 1;
    const bool reuse = b.use_cache && velver == 2 && *b.cache_epoch == *b.list_epoch &&
                       *b.cache_step == *b.step;
    __syncthreads();
    if (fill && blockIdx.x == 0 && threadIdx.x == 0) {
        *b.cache_epoch = *b.list_epoch;
        *b.cache_step = *b.step;
    }
    if (ONLY == 1 && !reuse) return;
    if (ONLY == 2 && reuse) return;
    if (ONLY != 2 && reuse) {
        for (long long base = next_warp_slots(b); base < b.N; base = next_warp_slots(b))
            force_fluid_slot_lean<R, true, DEPTH>(b, base + (threadIdx.x & 31), step, false, ring);
    } else if (ONLY != 1) {
        for (long long base = next_warp_slots(b); base < b.N; base = next_warp_slots(b))
            force_fluid_slot_lean<R, false, DEPTH>(b, base + (threadIdx.x & 31), step, fill, ring);
    }
}

// ONLY as in k_force_fluid_lean: 0 every path, 1 only the pass reading the
// cached normals, 2 only the drawing paths
template <class R, int ONLY = 0>
__global__ void __launch_bounds__(256) k_force_fluid(Bufs b, int velver)
{
    const uint32_t step = (uint32_t)(*b.step);
    const bool fill = b.use_cache && velver == 1;
    const bool reuse = b.use_cache && velver == 2 && *b.cache_epoch == *b.list_epoch &&
                       *b.cache_step == *b.step;
    // every warp reads the epochs before the first one is written below
    __syncthreads();
    if (fill && blockIdx.x == 0 && threadIdx.x == 0) {
        *b.cache_epoch = *b.list_epoch;
        *b.cache_step = *b.step;
    }
    // reuse is uniform over the launch
    if (ONLY == 1 && !reuse) return;
    if (ONLY == 2 && reuse) return;
    if (ONLY != 2 && reuse) {
        for (long long base = next_warp_slots(b); base < b.N; base = next_warp_slots(b))
            force_fluid_slot<R, true>(b, base + (threadIdx.x & 31), step, false);
    } else if (ONLY != 1) {
        for (long long base = next_warp_slots(b); base < b.N; base = next_warp_slots(b))
            force_fluid_slot<R, false>(b, base + (threadIdx.x & 31), step, fill);
    }
}

// ---------------------------------------------------- pair-stream force pass
// The direct pass (every pair from both sides) reorganised for the SIMT
// lanes: a warp owns 32 consecutive slots; phase A walks the 32 lists in
// step (the exact r < h decision, cheap) and compacts the surviving pairs
// into a ring in shared memory with ballots; phase B evaluates them 32 at a
// time -- Philox, Box-Muller and the SDPD pair of Eqs. FijC-FijT, or the
// fluid-sphere pair with the drag reaction -- with every lane busy whatever
// the spread of list lengths and of pairs beyond h; phase C hands each
// result back to the lane that owns the particle, which adds its pairs in
// list order.  The particle's own records are staged in shared memory for
// phase B.  The terms and their order are those of force_fluid_slot, so the
// forces equal the direct pass bit for bit.
template <class R> struct StreamSmem {
    using T4 = typename Vec<R>::T4;
    T4 qr[64];            // queued pairs: r_ij (x, y, z) and r^2
    T4 hB[32], hC[32], hD[32];   // records of the warp's own particles
    int2 qm[64];          // partner slot; entry k << 8 | owner lane << 1 | sphere partner
    int hinst[32];        // instance of each own particle
    R res[32 * 9];        // per batch position: f part (3), e x o (3), drag reaction (3)
};

template <class R, bool REUSE>
__device__ __forceinline__ void force_stream_group(const Bufs &b, StreamSmem<R> &S, long long base, uint32_t step,
                                                   bool fill)
{
    using T4 = typename Vec<R>::T4;
    using T2 = typename Vec2<R>::T2;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const long long s = base + lane;
    const long long Np = b.Npad;
    const T4 *__restrict__ A = Mir<R>::A(b);
    const T4 *__restrict__ Bm = Mir<R>::B(b);
    const T4 *__restrict__ Cm = Mir<R>::C(b);
    const T4 *__restrict__ Dm = Mir<R>::D(b);
    T4 *__restrict__ zA = (T4 *)b.zdA;
    T2 *__restrict__ zB = (T2 *)b.zdB;
    const bool mine = s < b.N && b.stype[s] == T_FLUID;
    int gi = 0, ii = 0, n = 0;
    T4 Ai;
    if (mine) {
        gi = b.perm[s];
        ii = b.pinst[gi];
        n = b.ncnt[s];
        Ai = A[s];
        S.hB[lane] = Bm[s];
        S.hC[lane] = Cm[s];
        S.hD[lane] = Dm[s];
    }
    S.hinst[lane] = ii;
    const Inst &I = b.inst[ii];
    const Geo<R> geo(I);
    PairK<R> P(I, step);        // constants of the instance of the pair in hand
    int pinst = ii;
    const bool own_fill = fill && P.noise;
    const R own_lev = P.lev;
    R fx = 0, fy = 0, fz = 0, tx = 0, ty = 0, tz = 0;
    uint64_t mask = 0;          // ring positions holding this lane's pairs
    unsigned head = 0, tail = 0;
    __syncwarp();

    // phase B + C on the ring positions [h0, h0 + cnt) (h0 a multiple of 32)
    auto batch = [&](unsigned h0, int cnt) {
        R g[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) g[c] = R(0);
        if (lane < cnt) {
            const unsigned p = (h0 + lane) & 63u;
            const T4 rq = S.qr[p];
            const int2 m = S.qm[p];
            const int j = m.x, k = m.y >> 8, il = (m.y >> 1) & 31;
            const bool rg = m.y & 1;
            const int pi = S.hinst[il];
            if (pi != pinst) {
                P = PairK<R>(b.inst[pi], step);
                pinst = pi;
            }
            const T4 Bi = S.hB[il], Ci = S.hC[il], Di = S.hD[il];
            const T4 Bj = Bm[j], Cj = Cm[j], Dj = Dm[j];
            const long long at = (long long)k * Np + base + il;
            Z6<R> z;
            int zmode = 0;
            if (REUSE && P.noise && !rg) {
                const T4 za = zA[at];
                const T2 zb = zB[at];
                if (!isnan(za.x)) {
                    z.z0 = za.x; z.z1 = za.y; z.z2 = za.z; z.z3 = za.w; z.z4 = zb.x; z.z5 = zb.y;
                    zmode = 1;
                }
            }
            R ox, oy, oz, ce, ex, ey, ez, q, om;
            sdpd_pair<R>(P, rq.x, rq.y, rq.z, rq.w, Bi, Ci, Di, Bj, Cj, Dj, !rg, zmode, z, ox, oy, oz, ce, ex, ey,
                         ez, q, om);
            if (!REUSE && fill && P.noise && !rg) {
                T4 zw;
                zw.x = z.z0; zw.y = z.z1; zw.z = z.z2; zw.w = z.z3;
                T2 zv;
                zv.x = z.z4; zv.y = z.z5;
                zA[at] = zw;
                zB[at] = zv;
            }
            pair_fh(ox, oy, oz, ce, ex, ey, ez, g[0], g[1], g[2], g[3], g[4], g[5]);
            if (rg) {
                R rcx, rcy, rcz;
                rxn_of(b, j, rcx, rcy, rcz);
                const R W = drag_weight(P, q, om);
                g[6] = mul_rn(rcx, W);
                g[7] = mul_rn(rcy, W);
                g[8] = mul_rn(rcz, W);
            }
#pragma unroll
            for (int c = 0; c < 9; ++c) S.res[lane * 9 + c] = g[c];
        }
        __syncwarp();
        // phase C: this lane's pairs of the batch, in ring (= list) order
        const unsigned off = h0 & 63u;
        uint32_t mm = (uint32_t)(mask >> off) & (cnt == 32 ? FULL : ((1u << cnt) - 1u));
        mask &= ~((uint64_t)mm << off);
        while (mm) {
            const int q = __ffs(mm) - 1;
            mm &= mm - 1;
            const R *rr = S.res + q * 9;
            // a zero drag-reaction term (non-sphere partner) leaves f unchanged exactly
            fx = sub_rn(fx, rr[6]);
            fy = sub_rn(fy, rr[7]);
            fz = sub_rn(fz, rr[8]);
            fx = add_rn(fx, rr[0]);
            fy = add_rn(fy, rr[1]);
            fz = add_rn(fz, rr[2]);
            tx = add_rn(tx, rr[3]);
            ty = add_rn(ty, rr[4]);
            tz = add_rn(tz, rr[5]);
        }
        __syncwarp();
    };

    // phase A: the lists in step, the next entry prefetched
    const int kmax = __reduce_max_sync(FULL, n);
    int jn = n > 0 ? __ldg(b.nbr + s) : 0;
    int jnn = n > 1 ? __ldg(b.nbr + Np + s) : 0;
    T4 An;
    if (n > 0) An = A[jn];
    for (int k = 0; k < kmax; ++k) {
        bool want = false, rig = false;
        int j = 0;
        R rx = 0, ry = 0, rz = 0, r2 = 0;
        if (k < n) {
            j = jn;
            const T4 Aj = An;
            if (k + 1 < n) {
                jn = jnn;
                An = A[jn];
                if (k + 2 < n) jnn = __ldg(b.nbr + (long long)(k + 2) * Np + s);
            }
            rig = mir_type(Aj) == T_RIGID;
            want = Rel<R>::get(b, I, geo, Ai, Aj, gi, j, rx, ry, rz, r2);
            if (!want && !REUSE && own_fill && !rig) {
                T4 nm;
                nm.x = R(NAN); nm.y = R(0); nm.z = R(0); nm.w = R(0);
                zA[(long long)k * Np + s] = nm;
            }
        }
        const unsigned bal = __ballot_sync(FULL, want);
        if (want) {
            const unsigned pos = (tail + __popc(bal & below)) & 63u;
            T4 rq;
            rq.x = rx; rq.y = ry; rq.z = rz; rq.w = r2;
            S.qr[pos] = rq;
            S.qm[pos] = make_int2(j, (k << 8) | (lane << 1) | (rig ? 1 : 0));
            mask |= 1ull << pos;
        }
        tail += __popc(bal);
        if (tail - head >= 32u) {
            __syncwarp();
            batch(head, 32);
            head += 32;
        }
    }
    if (tail != head) {   // fewer than 32 left
        __syncwarp();
        batch(head, (int)(tail - head));
    }
    if (mine) write_fluid_force<R>(b, I, gi, fx, fy, fz, tx, ty, tz, own_lev);
    __syncwarp();   // the smem of this group is reused by the next one
}

// MINB: resident 256-thread blocks per SM the registers are capped for (2:
// up to 128 registers, 16 warps; 3: 80 registers, 24 warps, a few spilled)
template <class R, int MINB>
__global__ void __launch_bounds__(256, MINB) k_force_stream(Bufs b, int velver)
{
    extern __shared__ __align__(32) unsigned char stream_smem[];
    StreamSmem<R> &S = reinterpret_cast<StreamSmem<R> *>(stream_smem)[threadIdx.x >> 5];
    const uint32_t step = (uint32_t)(*b.step);
    const bool fill = b.use_cache && velver == 1;
    const bool reuse = b.use_cache && velver == 2 && *b.cache_epoch == *b.list_epoch &&
                       *b.cache_step == *b.step;
    // every warp reads the epochs before the first one is written below
    __syncthreads();
    if (fill && blockIdx.x == 0 && threadIdx.x == 0) {
        *b.cache_epoch = *b.list_epoch;
        *b.cache_step = *b.step;
    }
    if (reuse) {
        for (long long base = next_warp_slots(b); base < b.N; base = next_warp_slots(b))
            force_stream_group<R, true>(b, S, base, step, false);
    } else {
        for (long long base = next_warp_slots(b); base < b.N; base = next_warp_slots(b))
            force_stream_group<R, false>(b, S, base, step, fill);
    }
}

// The direct pass with TPP lanes per particle (TPP = 2 or 4): the lanes of a
// particle take the entries sub, sub + TPP, ... of its list (sub = lane %
// TPP), each summing its share in list order, and a butterfly of shuffles
// adds the TPP partial sums in a fixed order; the first lane writes.  Small
// workloads so fill TPP times as many warps.
template <class R, bool REUSE, int TPP>
__device__ __forceinline__ void force_fluid_slot_tpp(const Bufs &b, long long s, int sub, uint32_t step, bool fill)
{
    using T4 = typename Vec<R>::T4;
    using T2 = typename Vec2<R>::T2;
    const bool active = s < b.N && b.stype[s] == T_FLUID;
    R fx = 0, fy = 0, fz = 0, tx = 0, ty = 0, tz = 0;
    int gi = 0;
    const Inst *Ip = b.inst;
    R lev = 0;
    if (active) {
        gi = b.perm[s];
        const Inst &I = b.inst[b.pinst[gi]];
        Ip = &I;
        const Geo<R> geo(I);
        const PairK<R> P(I, step);
        lev = P.lev;
        const bool fl = fill && P.noise;
        const T4 *__restrict__ A = Mir<R>::A(b);
        const T4 *__restrict__ Bm = Mir<R>::B(b);
        const T4 *__restrict__ Cm = Mir<R>::C(b);
        const T4 *__restrict__ Dm = Mir<R>::D(b);
        T4 *__restrict__ zA = (T4 *)b.zdA;
        T2 *__restrict__ zB = (T2 *)b.zdB;
        const int *__restrict__ nb = b.nbr + s;
        const T4 Ai = A[s], Bi = Bm[s], Ci = Cm[s], Di = Dm[s];
        const int n = b.ncnt[s];
        const long long Np = b.Npad;
        int jn = sub < n ? ld_stream(nb + (long long)sub * Np) : 0;
        int jnn = sub + TPP < n ? ld_stream(nb + (long long)(sub + TPP) * Np) : 0;
        T4 An = A[jn];
        T4 zan;
        T2 zbn;
        if (REUSE && P.noise && sub < n) {
            zan = ld_stream(zA + (long long)sub * Np + s);
            zbn = ld_stream(zB + (long long)sub * Np + s);
        }
        for (int k = sub; k < n; k += TPP) {
            const int j = jn;
            const T4 Aj = An;
            T4 za;
            T2 zb;
            if (REUSE) { za = zan; zb = zbn; }
            if (k + TPP < n) {
                jn = jnn;
                An = A[jn];
                if (REUSE && P.noise) {
                    zan = ld_stream(zA + (long long)(k + TPP) * Np + s);
                    zbn = ld_stream(zB + (long long)(k + TPP) * Np + s);
                }
                if (k + 2 * TPP < n) jnn = ld_stream(nb + (long long)(k + 2 * TPP) * Np);
            }
            const bool rig = mir_type(Aj) == T_RIGID;
            const long long at = (long long)k * Np + s;
            R rx, ry, rz, r2;
            if (!Rel<R>::get(b, I, geo, Ai, Aj, gi, j, rx, ry, rz, r2)) {
                if (!REUSE && fl && !rig) {
                    T4 nm;
                    nm.x = R(NAN); nm.y = R(0); nm.z = R(0); nm.w = R(0);
                    st_stream(zA + at, nm);
                }
                continue;
            }
            const T4 Bj = Bm[j], Cj = Cm[j], Dj = Dm[j];
            R ox, oy, oz, ce, ex, ey, ez, q, om;
            Z6<R> z;
            int zmode = 0;
            if (REUSE && P.noise && !rig && !isnan(za.x)) {
                z.z0 = za.x; z.z1 = za.y; z.z2 = za.z; z.z3 = za.w; z.z4 = zb.x; z.z5 = zb.y;
                zmode = 1;
            }
            sdpd_pair<R>(P, rx, ry, rz, r2, Bi, Ci, Di, Bj, Cj, Dj, !rig, zmode, z, ox, oy, oz, ce, ex, ey, ez,
                         q, om);
            if (!REUSE && fl && !rig) {
                T4 zw;
                zw.x = z.z0; zw.y = z.z1; zw.z = z.z2; zw.w = z.z3;
                T2 zv;
                zv.x = z.z4; zv.y = z.z5;
                st_stream(zA + at, zw);
                st_stream(zB + at, zv);
            }
            R gx, gy, gz, hx, hy, hz;
            pair_fh(ox, oy, oz, ce, ex, ey, ez, gx, gy, gz, hx, hy, hz);
            if (rig) {
                R rcx, rcy, rcz;
                rxn_of(b, j, rcx, rcy, rcz);
                const R W = drag_weight(P, q, om);
                fx = sub_rn(fx, mul_rn(rcx, W));
                fy = sub_rn(fy, mul_rn(rcy, W));
                fz = sub_rn(fz, mul_rn(rcz, W));
            }
            fx = add_rn(fx, gx);
            fy = add_rn(fy, gy);
            fz = add_rn(fz, gz);
            tx = add_rn(tx, hx);
            ty = add_rn(ty, hy);
            tz = add_rn(tz, hz);
        }
    }
    // the TPP lanes of the particle are consecutive: butterfly over them
#pragma unroll
    for (int o = 1; o < TPP; o <<= 1) {
        fx = add_rn(fx, __shfl_xor_sync(0xffffffffu, fx, o));
        fy = add_rn(fy, __shfl_xor_sync(0xffffffffu, fy, o));
        fz = add_rn(fz, __shfl_xor_sync(0xffffffffu, fz, o));
        tx = add_rn(tx, __shfl_xor_sync(0xffffffffu, tx, o));
        ty = add_rn(ty, __shfl_xor_sync(0xffffffffu, ty, o));
        tz = add_rn(tz, __shfl_xor_sync(0xffffffffu, tz, o));
    }
    if (active && sub == 0) write_fluid_force<R>(b, *Ip, gi, fx, fy, fz, tx, ty, tz, lev);
}

template <class R, int TPP>
__global__ void __launch_bounds__(256) k_force_fluid_tpp(Bufs b, int velver)
{
    const uint32_t step = (uint32_t)(*b.step);
    const bool fill = b.use_cache && velver == 1;
    const bool reuse = b.use_cache && velver == 2 && *b.cache_epoch == *b.list_epoch &&
                       *b.cache_step == *b.step;
    __syncthreads();
    if (fill && blockIdx.x == 0 && threadIdx.x == 0) {
        *b.cache_epoch = *b.list_epoch;
        *b.cache_step = *b.step;
    }
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(b.work, (unsigned long long)(32 / TPP));
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((long long)base >= b.N) break;
        const long long s = (long long)base + lane / TPP;
        if (reuse) force_fluid_slot_tpp<R, true, TPP>(b, s, lane % TPP, step, false);
        else force_fluid_slot_tpp<R, false, TPP>(b, s, lane % TPP, step, fill);
    }
}

// Newton-3 force pass, phase 1: every fluid or wall particle evaluates the
// pairs of its owned prefix (see k_neighbors; within h, both non-rigid, at
// least one fluid) once, stores (f, e x o) in the partner's column of the
// pair buffer (at the row of the partner's entry for the pair, from k_rev)
// and keeps its own sum.  Each unordered pair is
// computed once instead of twice.  The first evaluation of a step stores the
// six normals of each pair; the second reads them back, fetched one entry
// ahead like the records, when the list has not been rebuilt in between (same
// counter, so the same bits).
// PUSH: the owner writes the finished pair result {f, e x o} into the
// partner's column (FP64, and FP32 in force mode 4); otherwise (FP32, mode 1)
// it keeps {o, ce} in its own column and the partner rebuilds f and e x o.
// Both hand the partner the same bits.
template <class R, bool REUSE, bool PUSH>
__device__ __forceinline__ void force_half_slot(const Bufs &b, long long s, uint32_t step, bool fill)
{
    using T4 = typename Vec<R>::T4;
    using T2 = typename Vec2<R>::T2;
    if (s >= b.N) return;
    const int ti = b.stype[s];
    if (ti == T_RIGID) return;
    const int gi = b.perm[s];
    const Inst &I = b.inst[b.pinst[gi]];
    const Geo<R> geo(I);
    const PairK<R> P(I, step);
    const T4 *__restrict__ A = Mir<R>::A(b);
    const T4 *__restrict__ Bm = Mir<R>::B(b);
    const T4 *__restrict__ Cm = Mir<R>::C(b);
    const T4 *__restrict__ Dm = Mir<R>::D(b);
    T4 *__restrict__ resA = (T4 *)b.resA;
    T2 *__restrict__ resB = (T2 *)b.resB;
    T4 *__restrict__ zA = (T4 *)b.zA;
    T2 *__restrict__ zB = (T2 *)b.zB;
    const int *__restrict__ nb = b.nbr + s;
    const uint16_t *__restrict__ rv = b.rev + s;
    const T4 Ai = A[s], Bi = Bm[s], Ci = Cm[s], Di = Dm[s];
    const bool fi = (ti == T_FLUID);
    R fx = 0, fy = 0, fz = 0, tx = 0, ty = 0, tz = 0;
    const int last = b.nfirst[s];  // the owned prefix of the list
    const long long Np = b.Npad;
    const bool noise = P.noise;
    int jn = 0 < last ? __ldg(nb) : 0;
    int jnn = 1 < last ? __ldg(nb + Np) : 0;
    T4 An = A[jn], Bn = Bm[jn], Cn = Cm[jn], Dn = Dm[jn];
    T4 zan;
    T2 zbn;
    if (REUSE && noise && last > 0) { zan = zA[s]; zbn = zB[s]; }
    for (int k = 0; k < last; ++k) {
        const int j = jn;
        const T4 Aj = An, Bj = Bn, Cj = Cn, Dj = Dn;
        T4 za;
        T2 zb;
        if (REUSE) { za = zan; zb = zbn; }
        if (k + 1 < last) {
            jn = jnn;
            An = A[jn]; Bn = Bm[jn]; Cn = Cm[jn]; Dn = Dm[jn];
            if (REUSE && noise) {
                zan = zA[(long long)(k + 1) * Np + s];
                zbn = zB[(long long)(k + 1) * Np + s];
            }
            if (k + 2 < last) jnn = __ldg(nb + (long long)(k + 2) * Np);
        }
        const int tj = mir_type(Aj);
        if (tj == T_RIGID) {
            if (fi) fluid_rigid_pair<R>(b, I, geo, P, gi, Ai, Bi, Ci, Di, j, Aj, Bj, Cj, Dj, fx, fy, fz, tx,
                                        ty, tz);
            continue;
        }
        if (!fi && tj != T_FLUID) continue;
        const long long at = (long long)k * Np + s;   // own column: normals cache
        // FP64 results go to the partner's column, at the row of its entry
        // for this pair (from k_rev); split results stay in the own column
        long long pt = at;
        bool put = true;
        if constexpr (PUSH) {
            const int row = __ldg(rv + (long long)k * Np);
            put = row < b.capown;   // false only after a list error (flagged)
            pt = (long long)row * Np + j;
        }
        R rx, ry, rz, r2;
        if (!Rel<R>::get(b, I, geo, Ai, Aj, gi, j, rx, ry, rz, r2)) {
            // beyond h: marked for the partner's gather and the normals cache
            T4 nm;
            nm.x = R(NAN); nm.y = R(0); nm.z = R(0); nm.w = R(0);
            if (put) resA[pt] = nm;
            if (!REUSE && fill) zA[at] = nm;
            continue;
        }
        Z6<R> z;
        int zmode = 0;
        // an entry beyond h in the first evaluation carries the NaN marker
        if (REUSE && noise && !isnan(za.x)) {
            z.z0 = za.x; z.z1 = za.y; z.z2 = za.z; z.z3 = za.w; z.z4 = zb.x; z.z5 = zb.y;
            zmode = 1;
        }
        R ox, oy, oz, ce, ex, ey, ez, q, om;
        sdpd_pair<R>(P, rx, ry, rz, r2, Bi, Ci, Di, Bj, Cj, Dj, true, zmode, z, ox, oy, oz, ce, ex, ey,
                     ez, q, om);
        if (!REUSE && fill && noise) {
            T4 zw;
            zw.x = z.z0; zw.y = z.z1; zw.z = z.z2; zw.w = z.z3;
            T2 zv;
            zv.x = z.z4; zv.y = z.z5;
            zA[at] = zw;
            zB[at] = zv;
        }
        R gx, gy, gz, hx, hy, hz;
        pair_fh(ox, oy, oz, ce, ex, ey, ez, gx, gy, gz, hx, hy, hz);
        T4 ra;
        if constexpr (!PUSH) {
            // {o, ce} (16 B); the partner rebuilds f and e x o
            ra.x = ox; ra.y = oy; ra.z = oz; ra.w = ce;
        } else {
            ra.x = gx; ra.y = gy; ra.z = gz; ra.w = hx;
            T2 rb;
            rb.x = hy; rb.y = hz;
            if (put) resB[pt] = rb;
        }
        if (put) resA[pt] = ra;
        fx += gx; fy += gy; fz += gz;
        tx += hx; ty += hy; tz += hz;
    }
    if (fi) {
        T4 oa;
        oa.x = fx; oa.y = fy; oa.z = fz; oa.w = tx;
        T2 ob;
        ob.x = ty; ob.y = tz;
        ((T4 *)b.ownA)[s] = oa;
        ((T2 *)b.ownB)[s] = ob;
    }
}

// (FP32: at most 128 registers, so four 128-thread blocks fit on an SM)
template <class R, bool PUSH>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1) k_force_half(Bufs b, int velver)
{
    const uint32_t step = (uint32_t)(*b.step);
    const bool fill = b.use_cache && velver == 1;
    const bool reuse = b.use_cache && velver == 2 && *b.cache_epoch == *b.list_epoch &&
                       *b.cache_step == *b.step;
    // every warp reads the epochs before the first one is written below
    __syncthreads();
    if (fill && blockIdx.x == 0 && threadIdx.x == 0) {
        *b.cache_epoch = *b.list_epoch;
        *b.cache_step = *b.step;
    }
    // reuse is uniform over the launch
    if (reuse) {
        for (long long base = next_warp_slots(b); base < b.N; base = next_warp_slots(b))
            force_half_slot<R, true, PUSH>(b, base + (threadIdx.x & 31), step, false);
    } else {
        for (long long base = next_warp_slots(b); base < b.N; base = next_warp_slots(b))
            force_half_slot<R, false, PUSH>(b, base + (threadIdx.x & 31), step, fill);
    }
}

// Newton-3 force pass, phase 2 (fluid particles): own sum + the results of
// the pairs its partners own (force negated, e x o equal; pairs the owner
// found beyond h carry a NaN marker) + the pairs with rigid neighbours among
// the non-owned entries, evaluated here (Eqs. FijC, FijD and the drag
// reaction Eq. F_fpi_DG_reac), all in entry order + external force.  FP64
// results were written into this particle's column (read coalesced); split
// results are read from the owner's column through the reverse index.
template <class R, bool PUSH>
__global__ void __launch_bounds__(256) k_force_gather(Bufs b)
{
    using T4 = typename Vec<R>::T4;
    using T2 = typename Vec2<R>::T2;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.N) return;
    if (b.stype[s] != T_FLUID) return;
    const int gi = b.perm[s];
    const Inst &I = b.inst[b.pinst[gi]];
    const Geo<R> geo(I);
    const T4 *__restrict__ A = Mir<R>::A(b);
    const T4 *__restrict__ resA = (const T4 *)b.resA;
    const T2 *__restrict__ resB = (const T2 *)b.resB;
    const int *__restrict__ nb = b.nbr + s;
    const uint16_t *__restrict__ rv = b.rev + s;
    const T4 Ai = A[s];
    const T4 oa = ((const T4 *)b.ownA)[s];
    const T2 ob = ((const T2 *)b.ownB)[s];
    R fx = oa.x, fy = oa.y, fz = oa.z, tx = oa.w, ty = ob.x, tz = ob.y;
    const int n = b.ncnt[s], first = b.nfirst[s];
    const long long Np = b.Npad;
    const bool any_rigid = b.nbflag[s] & 1;
    // more non-owned entries than capown only after a list error (flagged)
    const int nend = min(n, first + b.capown);
    constexpr int G = 4;
    for (int k0 = first; k0 < nend; k0 += G) {
        long long at[G];
        int pj[G];
        bool use[G], rig[G];
        T4 Ap[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int k = k0 + g;
            use[g] = k < nend;
            rig[g] = false;
            const int i = use[g] ? __ldg(nb + (long long)k * Np) : 0;
            pj[g] = i;
            if (use[g] && (!PUSH || any_rigid)) {
                Ap[g] = A[i];
                rig[g] = mir_type(Ap[g]) == T_RIGID;
            }
            if constexpr (PUSH) at[g] = (long long)(k - first) * Np + s;
            else at[g] = (long long)(use[g] ? __ldg(rv + (long long)k * Np) : 0) * Np + i;
        }
        T4 ra[G];
        T2 rb[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (use[g] && !rig[g]) {
                ra[g] = resA[at[g]];
                if constexpr (PUSH) rb[g] = resB[at[g]];
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (!use[g]) continue;
            if (rig[g]) {
                R f[6] = { fx, fy, fz, tx, ty, tz };
                fluid_rigid_pair_call<R>(b, s, gi, pj[g], f);
                fx = f[0]; fy = f[1]; fz = f[2]; tx = f[3]; ty = f[4]; tz = f[5];
                continue;
            }
            // NaN marks a pair beyond h (written by the owner)
            if (isnan(ra[g].x)) continue;
            if constexpr (PUSH) {
                fx -= ra[g].x; fy -= ra[g].y; fz -= ra[g].z;
                tx += ra[g].w; ty += rb[g].x; tz += rb[g].y;
            } else {
                // e of the owner = -(e seen from here), bitwise
                R rx, ry, rz;
                geo.disp(Ai, Ap[g], rx, ry, rz);
                const R ir = rsqrt_<R>(rx * rx + ry * ry + rz * rz);
                R gx, gy, gz, hx, hy, hz;
                pair_fh(ra[g].x, ra[g].y, ra[g].z, ra[g].w, -(rx * ir), -(ry * ir), -(rz * ir), gx, gy, gz,
                        hx, hy, hz);
                fx -= gx; fy -= gy; fz -= gz;
                tx += hx; ty += hy; tz += hz;
            }
        }
    }
    write_fluid_force<R>(b, I, gi, fx, fy, fz, tx, ty, tz, K<R>::lever(I));
}

// -------------------------------------------------------- rigid force pass
__device__ __forceinline__ void cross3(const double a[3], const double c[3], double o[3])
{
    o[0] = a[1] * c[2] - a[2] * c[1];
    o[1] = a[2] * c[0] - a[0] * c[2];
    o[2] = a[0] * c[1] - a[1] * c[0];
}

__device__ __forceinline__ void dem_coeffs(const Inst &I, double Ri, double Rj, double mi, double mj,
                                           double &kn, double &kt, double &cn, double &ct)
{
    const double ms = (mj > 0.0) ? mi * mj / (mi + mj) : mi;
    if (I.dem_law == 0) {
        const double D = (1.0 - I.nu_p * I.nu_p) / (I.E_p * PI);
        const double Re = (Rj > 0.0) ? Ri * Rj / (Ri + Rj) : Ri;
        kn = 4.0 / (3.0 * PI) * (1.0 / (D + D)) * sqrt(Re);
        kt = kn * I.kt_ratio;
        cn = 2.0 * sqrt(2.0 * ms * kn);
        ct = 2.0 * sqrt(2.0 * ms * kt);
    } else {
        kn = I.kn;
        kt = kn * I.kt_ratio;
        cn = 2.0 * I.zeta * sqrt(ms * kn);
        ct = 2.0 * I.zeta * sqrt(ms * kt);
    }
}

// One DEM contact on rigid particle i (n from the partner to i, overlap < 0):
// normal spring-dashpot, tangential spring-dashpot on the stored displacement
// with the Coulomb slider, torque (-R_i n) x F; also the next tangential
// displacement |delta| t + v_t dt, capped at the slider limit (dn).
__device__ void dem_pair(const Bufs &b, const Inst &I, int r, int partner, const double n[3],
                         double overlap, const double vij[3], const double wsR[3], double Ri,
                         double kn, double kt, double cn, double ct, double F[3], double T[3],
                         double dn[3])
{
    const double vn = vij[0] * n[0] + vij[1] * n[1] + vij[2] * n[2];
    double Fn[3], wxn[3], vt[3];
    cross3(wsR, n, wxn);
    for (int a = 0; a < 3; ++a) {
        Fn[a] = -kn * overlap * n[a] - cn * vn * n[a];
        vt[a] = vij[a] - vn * n[a] - wxn[a];
    }
    double dl[3] = { 0.0, 0.0, 0.0 };
    const int K = b.K;
    const int hc = b.h_n[r];
    for (int k = 0; k < hc; ++k)
        if (b.h_part[r * K + k] == partner) {
            for (int a = 0; a < 3; ++a) dl[a] = b.h_del[((long long)r * K + k) * 3 + a];
            break;
        }
    const double vtm = sqrt(vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]);
    const double dm = sqrt(dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2]);
    double t[3] = { 0.0, 0.0, 0.0 };
    if (vtm > 0.0) {
        for (int a = 0; a < 3; ++a) t[a] = vt[a] / vtm;
    } else if (dm > 0.0) {
        for (int a = 0; a < 3; ++a) t[a] = dl[a] / dm;
    }
    double Ft[3];
    for (int a = 0; a < 3; ++a) Ft[a] = -kt * dl[a] - ct * vt[a];
    const double Fnm = sqrt(Fn[0] * Fn[0] + Fn[1] * Fn[1] + Fn[2] * Fn[2]);
    const double Ftm = sqrt(Ft[0] * Ft[0] + Ft[1] * Ft[1] + Ft[2] * Ft[2]);
    if (Ftm >= I.mu_fric * Fnm)
        for (int a = 0; a < 3; ++a) Ft[a] = -I.mu_fric * Fnm * t[a];
    double Fs[3], lev[3], tq[3];
    for (int a = 0; a < 3; ++a) {
        Fs[a] = Fn[a] + Ft[a];
        lev[a] = -Ri * n[a];
    }
    cross3(lev, Fs, tq);
    for (int a = 0; a < 3; ++a) {
        F[a] += Fs[a];
        T[a] += tq[a];
    }
    for (int a = 0; a < 3; ++a) dn[a] = dm * t[a] + vt[a] * I.dt;
    const double dnm = sqrt(dn[0] * dn[0] + dn[1] * dn[1] + dn[2] * dn[2]);
    const double cap = kt > 0.0 ? I.mu_fric * Fnm / kt : 0.0;
    if (dnm > cap && dnm > 0.0) {
        const double sc = cap / dnm;
        for (int a = 0; a < 3; ++a) dn[a] *= sc;
    }
}

__device__ __forceinline__ void hist_put(const Bufs &b, int r, int slot, int partner, const double dn[3])
{
    if (slot < b.K) {
        b.hn_part[r * b.K + slot] = partner;
        for (int a = 0; a < 3; ++a) b.hn_del[((long long)r * b.K + slot) * 3 + a] = dn[a];
    } else {
        atomicOr(b.err, ERR_CONTACT_CAP);
    }
}

// Rigid particles, one warp each: pressure-gradient force from the fluid
// neighbours (Eq. F_fpi_PG), DEM + lubrication with the rigid neighbours,
// wall planes, drag, gravity.  The lanes take the neighbour list in rounds of
// 32 for the fluid pairs and collect the rigid entries, in list order, in
// shared memory.  A sphere has only a few sphere neighbours, so the block's
// RPB spheres pool theirs: the pooled pairs run one per thread, RB at a time
// (their FP64 DEM and lubrication arithmetic on every lane instead of on a
// few lanes of each warp), each result is kept in shared memory, and each
// sphere adds its own in list order.  New history entries go to slots in list
// order, so the table is deterministic.
struct RigidPairRes {
    double F[3], T[3], L[3], dn[3];   // DEM force and torque, lubrication, next tangential displacement
    int partner;                      // gid of a contact partner, -1 without contact
    int pad;
};
__host__ __device__ inline size_t rigid_list_bytes(int cap) { return ((size_t)RPB * cap * sizeof(uint32_t) + 15) / 16 * 16; }
__host__ __device__ inline size_t rigid_smem_bytes(int cap) { return rigid_list_bytes(cap) + (size_t)RB * sizeof(RigidPairRes); }

template <class R>
__global__ void __launch_bounds__(RB) k_force_rigid(Bufs b, int velver)
{
    extern __shared__ __align__(16) unsigned char rsm[];
    __shared__ double s_x[RPB][3], s_v[RPB][3], s_w[RPB][3], s_R[RPB], s_m[RPB];
    __shared__ int s_r[RPB], s_inst[RPB], s_nr[RPB], s_pre[RPB + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * RPB + warp;
    const bool live = r < b.nrigid;   // a warp past the end only takes part in the barriers
    uint32_t *const lists = reinterpret_cast<uint32_t *>(rsm);
    uint32_t *rl = lists + (size_t)warp * b.cap;   // this warp's rigid entries
    RigidPairRes *pres = reinterpret_cast<RigidPairRes *>(rsm + rigid_list_bytes(b.cap));
    const int g = live ? b.rigid_gid[r] : 0;
    const long long s = live ? b.slot_of[g] : 0;
    const Inst &I = b.inst[b.pinst[g]];
    double xi[3] = { 0.0, 0.0, 0.0 }, vi[3] = { 0.0, 0.0, 0.0 }, wi[3] = { 0.0, 0.0, 0.0 };
    double Ri = 0.0, mi = 0.0, di = 0.0;
    if (live) {
        for (int a = 0; a < 3; ++a) {
            xi[a] = b.x[3 * g + a];
            vi[a] = b.v[3 * g + a];
            wi[a] = b.w[3 * g + a];
        }
        Ri = b.R[g];
        mi = b.m[g];
        di = b.sd[s];
        if (lane == 0) {
            for (int a = 0; a < 3; ++a) {
                s_x[warp][a] = xi[a];
                s_v[warp][a] = vi[a];
                s_w[warp][a] = wi[a];
            }
            s_R[warp] = Ri;
            s_m[warp] = mi;
            s_r[warp] = r;
            s_inst[warp] = b.pinst[g];
        }
    }
    const bool commit = (velver == 2);
    const long long Np = b.Npad;
    double acc[15];
#pragma unroll
    for (int a = 0; a < 15; ++a) acc[a] = 0.0;   // pg, npg, Fdem, Tdem, Flub
    // the fluid pairs in precision R on the mirrors, as for fluid pairs (the
    // C + D part of the SDPD pair, the exact r < h decision of Rel), summed
    // per lane in R; DEM and lubrication stay FP64
    using T4 = typename Vec<R>::T4;
    const PairK<R> P(I, 0u);
    const Geo<R> geo(I);
    const T4 *__restrict__ A = Mir<R>::A(b);
    const T4 *__restrict__ Bm = Mir<R>::B(b);
    const T4 *__restrict__ Cm = Mir<R>::C(b);
    const T4 *__restrict__ Dm = Mir<R>::D(b);
    const T4 Ai = A[s], Bi = Bm[s], Ci = Cm[s], Di = Dm[s];
    const R Rr = (R)Ri;
    R f0 = 0, f1 = 0, f2 = 0, t0 = 0, t1 = 0, t2 = 0;
    const int n = live ? b.ncnt[s] : 0;
    const unsigned below = (1u << lane) - 1u;
    int nr = 0;   // rigid entries collected
    // the entry of the next round is fetched one round ahead
    uint32_t en = lane < n ? (uint32_t)__ldg(b.nbr + (long long)lane * Np + s) : 0u;
    for (int kk = 0; kk < n; kk += 32) {
        const int k = kk + lane;
        bool rig = false;
        const uint32_t e = en;
        if (k + 32 < n) en = (uint32_t)__ldg(b.nbr + (long long)(k + 32) * Np + s);
        if (k < n) {
            const int j = (int)(e & ~NB_FAR);
            const T4 Aj = A[j];
            const int tj = mir_type(Aj);
            if (tj == T_FLUID && !(e & NB_FAR)) {
                // F^C + F^D of the pair (s, j), summed for Eq. F_fpi_PG
                R rx, ry, rz, r2;
                if (Rel<R>::get(b, I, geo, Ai, Aj, g, j, rx, ry, rz, r2)) {
                    Z6<R> z;
                    R ox, oy, oz, ce, ex, ey, ez, q, om;
                    sdpd_pair<R>(P, rx, ry, rz, r2, Bi, Ci, Di, Bm[j], Cm[j], Dm[j], false, 0, z, ox, oy, oz, ce,
                                 ex, ey, ez, q, om);
                    f0 += ox + ce * ex;
                    f1 += oy + ce * ey;
                    f2 += oz + ce * ez;
                    // lever -R e: (-R e) x (o + ce e) = -R e x o
                    t0 -= Rr * (ey * oz - ez * oy);
                    t1 -= Rr * (ez * ox - ex * oz);
                    t2 -= Rr * (ex * oy - ey * ox);
                }
            } else {
                rig = (tj == T_RIGID);
            }
        }
        const unsigned rb = __ballot_sync(0xffffffffu, rig);
        if (rig) rl[nr + __popc(rb & below)] = e;
        nr += __popc(rb);
    }
    if (lane == 0) s_nr[warp] = nr;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_pre[0] = 0;
        for (int w = 0; w < RPB; ++w) s_pre[w + 1] = s_pre[w] + s_nr[w];
    }
    __syncthreads();
    // the pooled rigid pairs (sphere w's entries at [s_pre[w], s_pre[w+1])),
    // RB at a time: DEM contact, or lubrication
    const int total = s_pre[RPB];
    double mine = 0.0;   // lane c < 9 of a live warp: component c of F_dem, T_dem, F_lub
    int base = 0;        // history slots used so far (the same on every lane)
    for (int c0 = 0; c0 < total; c0 += RB) {
        const int p = c0 + threadIdx.x;
        if (p < total) {
            int ws = 0;
            while (ws + 1 < RPB && s_pre[ws + 1] <= p) ++ws;
            const uint32_t e = lists[(size_t)ws * b.cap + (p - s_pre[ws])];
            const Inst &Iw = b.inst[s_inst[ws]];
            const double xs[3] = { s_x[ws][0], s_x[ws][1], s_x[ws][2] };
            const double Rs = s_R[ws];
            RigidPairRes &o = pres[threadIdx.x];
            for (int a = 0; a < 3; ++a) {
                o.F[a] = 0.0;
                o.T[a] = 0.0;
                o.L[a] = 0.0;
                o.dn[a] = 0.0;
            }
            o.partner = -1;
            const int j = (int)(e & ~NB_FAR);
            const int gj = b.perm[j];
            const double xj[3] = { b.x[3 * gj], b.x[3 * gj + 1], b.x[3 * gj + 2] };
            double rv[3];
            const double r2 = exact_disp(xs, xj, Iw, rv);
            const double L = sqrt(r2);
            const double vij[3] = { s_v[ws][0] - b.v[3 * gj], s_v[ws][1] - b.v[3 * gj + 1],
                                    s_v[ws][2] - b.v[3 * gj + 2] };
            const double Rj = b.R[gj];
            const double dsum = Rs + Rj;
            if (L < dsum) {
                const double nn[3] = { rv[0] / L, rv[1] / L, rv[2] / L };
                double wsR[3];
                for (int a = 0; a < 3; ++a) wsR[a] = Rs * s_w[ws][a] + Rj * b.w[3 * gj + a];
                double kn, kt, cn, ct;
                dem_coeffs(Iw, Rs, Rj, s_m[ws], b.m[gj], kn, kt, cn, ct);
                dem_pair(b, Iw, s_r[ws], gj, nn, L - dsum, vij, wsR, Rs, kn, kt, cn, ct, o.F, o.T, o.dn);
                o.partner = gj;
            } else if (r2 < Iw.rc2) {
                double gap = L - dsum;
                const double gmin = Iw.lub_gap_min * dsum;
                if (gap < gmin) gap = gmin;
                const double c = 3.0 * PI * Iw.eta * dsum * dsum / (8.0 * gap);
                for (int a = 0; a < 3; ++a) o.L[a] = c * (-vij[a]);
            }
        }
        __syncthreads();
        // each sphere adds its own pairs of this chunk in list order
        if (live) {
            const int lo = max(s_pre[warp], c0) - c0, hi = min(s_pre[warp + 1], c0 + RB) - c0;
            for (int t = lo; t < hi; ++t) {
                const RigidPairRes &o = pres[t];
                if (lane < 9) mine += lane < 3 ? o.F[lane] : (lane < 6 ? o.T[lane - 3] : o.L[lane - 6]);
                if (o.partner >= 0) {
                    if (lane == 0 && commit) hist_put(b, r, base, o.partner, o.dn);
                    ++base;
                }
            }
        }
        __syncthreads();
    }
    if (!live) return;   // past the block's last barrier
    acc[0] = f0; acc[1] = f1; acc[2] = f2;
    acc[3] = t0; acc[4] = t1; acc[5] = t2;
#pragma unroll
    for (int a = 0; a < 6; ++a) acc[a] = warp_sum(acc[a]);
#pragma unroll
    for (int c = 0; c < 9; ++c) acc[6 + c] = __shfl_sync(0xffffffffu, mine, c);
    if (lane != 0) return;
    // contact with the planes bounding the domain on wall axes
    for (int a = 0; a < 3; ++a) {
        if (I.periodic[a]) continue;
        for (int side = 0; side < 2; ++side) {
            const double L = side == 0 ? xi[a] - I.origin[a] : (I.origin[a] + I.box[a]) - xi[a];
            if (!(L < Ri)) continue;
            double nn[3] = { 0, 0, 0 };
            nn[a] = side == 0 ? 1.0 : -1.0;
            double wsR[3], dn[3];
            for (int c = 0; c < 3; ++c) wsR[c] = Ri * wi[c];
            double kn, kt, cn, ct;
            dem_coeffs(I, Ri, 0.0, mi, 0.0, kn, kt, cn, ct);
            dem_pair(b, I, r, PLANE_BASE + 2 * a + side, nn, L - Ri, vi, wsR, Ri, kn, kt, cn, ct,
                     acc + 6, acc + 9, dn);
            if (commit) hist_put(b, r, base, PLANE_BASE + 2 * a + side, dn);
            ++base;
        }
    }
    if (commit) b.hn_n[r] = base < b.K ? base : b.K;
    const double Vs = 4.0 / 3.0 * PI * Ri * Ri * Ri;
    const double sc = Vs * di;
    double ax[3];
    ext_accel(I, xi, ax);
    for (int a = 0; a < 3; ++a) {
        b.F[3 * g + a] = sc * acc[a] + b.fdg[3 * r + a] + acc[6 + a] + acc[12 + a] + mi * ax[a];
        b.T[3 * g + a] = sc * acc[3 + a] + acc[9 + a];
    }
}

__global__ void k_hist_copy(Bufs b)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= b.nrigid) return;
    const int n = b.hn_n[r];
    b.h_n[r] = n;
    for (int k = 0; k < n; ++k) {
        b.h_part[r * b.K + k] = b.hn_part[r * b.K + k];
        for (int a = 0; a < 3; ++a)
            b.h_del[((long long)r * b.K + k) * 3 + a] = b.hn_del[((long long)r * b.K + k) * 3 + a];
    }
}

// ---------------------------------------------------------------- launchers
static inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// Blocks of a persistent launch: as many as are resident at once (never
// more than the warps needed to cover N).
template <class K>
static unsigned persistent_grid(K kernel, int block, long long N)
{
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long need = (N + block - 1) / block;
    return (unsigned)std::min<long long>(need, (long long)nsm * per_sm);
}

void launch_density(const Bufs &b, int precision, int dflags, int newton3, const int *gate, cudaStream_t st)
{
    if (!b.N) return;
    const int any_filter = dflags & 1, any_reinit = (dflags >> 1) & 1, any_artvis = (dflags >> 2) & 1;
    // the density kernels leave the mirrors to a later pass when one follows
    const int defer = any_filter | any_reinit;
    if (precision == SDPD_PREC_FP64 && newton3) {
        cudaMemsetAsync(b.work, 0, sizeof(unsigned long long), st);
        k_density_half<<<persistent_grid(k_density_half, b.pair_block, b.N), b.pair_block, 0, st>>>(b, gate);
        k_density_gather<<<nblk(b.N, b.pair_block), b.pair_block, 0, st>>>(b, defer, gate);
        if (any_reinit) {
            k_reinit<double><<<nblk(b.N, b.pair_block), b.pair_block, 0, st>>>(b, any_filter, gate);
            k_reinit_copy<<<nblk(b.N, 256), 256, 0, st>>>(b, gate);
        }
        if (any_filter) k_filter<double><<<nblk(b.N, b.pair_block), b.pair_block, 0, st>>>(b, gate);
    } else if (precision == SDPD_PREC_SPLIT) {
        if (any_artvis) k_density<float, true><<<nblk(b.N, b.pair_block), b.pair_block, 0, st>>>(b, defer, gate);
        else k_density<float, false><<<nblk(b.N, b.pair_block), b.pair_block, 0, st>>>(b, defer, gate);
        if (any_reinit) {
            k_reinit<float><<<nblk(b.N, b.pair_block), b.pair_block, 0, st>>>(b, any_filter, gate);
            k_reinit_copy<<<nblk(b.N, 256), 256, 0, st>>>(b, gate);
        }
        if (any_filter) k_filter<float><<<nblk(b.N, b.pair_block), b.pair_block, 0, st>>>(b, gate);
    } else {
        if (any_artvis) k_density<double, true><<<nblk(b.N, b.pair_block), b.pair_block, 0, st>>>(b, defer, gate);
        else k_density<double, false><<<nblk(b.N, b.pair_block), b.pair_block, 0, st>>>(b, defer, gate);
        if (any_reinit) {
            k_reinit<double><<<nblk(b.N, b.pair_block), b.pair_block, 0, st>>>(b, any_filter, gate);
            k_reinit_copy<<<nblk(b.N, 256), 256, 0, st>>>(b, gate);
        }
        if (any_filter) k_filter<double><<<nblk(b.N, b.pair_block), b.pair_block, 0, st>>>(b, gate);
    }
}

void launch_drag(const Bufs &b, int precision, cudaStream_t st)
{
    if (!b.nrigid) return;
    const unsigned g = nblk(b.nrigid, RPB);
    if (precision == SDPD_PREC_SPLIT) k_drag<float><<<g, RB, 0, st>>>(b);
    else k_drag<double><<<g, RB, 0, st>>>(b);
    k_drag_law<<<nblk(b.nrigid, 64), 64, 0, st>>>(b);
}


template <class R>
static size_t stream_smem_bytes(int block) { return (size_t)(block / 32) * sizeof(StreamSmem<R>); }

void init_pair_kernels()
{
    // the sphere kernel's rigid lists and pooled-pair results at the largest
    // list capacity
    cudaFuncSetAttribute(k_force_rigid<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)rigid_smem_bytes(SDPD_MAX_NEIGHBORS));
    cudaFuncSetAttribute(k_force_rigid<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)rigid_smem_bytes(SDPD_MAX_NEIGHBORS));
    // the pair-stream kernels' shared memory at the largest block (256)
    cudaFuncSetAttribute(k_force_stream<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)stream_smem_bytes<float>(256));
    cudaFuncSetAttribute(k_force_stream<float, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)stream_smem_bytes<float>(256));
    cudaFuncSetAttribute(k_force_stream<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)stream_smem_bytes<double>(256));
}

template <class K>
static unsigned persistent_grid_smem(K kernel, int block, size_t smem, long long N)
{
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long need = (N + block - 1) / block;
    return (unsigned)std::min<long long>(need, (long long)nsm * per_sm);
}

void launch_forces(const Bufs &b, int precision, int velver, int newton3, cudaStream_t st)
{
    if (!b.N) return;
    const int bs = b.pair_block;
    cudaMemsetAsync(b.work, 0, sizeof(unsigned long long), st);
    if (newton3 == 2 || newton3 == 3) {
        if (precision == SDPD_PREC_SPLIT) {
            const size_t sm = stream_smem_bytes<float>(bs);
            if (newton3 == 3)
                k_force_stream<float, 3>
                    <<<persistent_grid_smem(k_force_stream<float, 3>, bs, sm, b.N), bs, sm, st>>>(b, velver);
            else
                k_force_stream<float, 2>
                    <<<persistent_grid_smem(k_force_stream<float, 2>, bs, sm, b.N), bs, sm, st>>>(b, velver);
        } else {
            const size_t sm = stream_smem_bytes<double>(bs);
            k_force_stream<double, 1>
                <<<persistent_grid_smem(k_force_stream<double, 1>, bs, sm, b.N), bs, sm, st>>>(b, velver);
        }
    } else if (newton3 == 1 || newton3 == 4) {
        if (precision == SDPD_PREC_SPLIT && newton3 == 4) {
            k_force_half<float, true><<<persistent_grid(k_force_half<float, true>, bs, b.N), bs, 0, st>>>(b, velver);
            k_force_gather<float, true><<<nblk(b.N, bs), bs, 0, st>>>(b);
        } else if (precision == SDPD_PREC_SPLIT) {
            k_force_half<float, false><<<persistent_grid(k_force_half<float, false>, bs, b.N), bs, 0, st>>>(b, velver);
            k_force_gather<float, false><<<nblk(b.N, bs), bs, 0, st>>>(b);
        } else {
            k_force_half<double, true><<<persistent_grid(k_force_half<double, true>, bs, b.N), bs, 0, st>>>(b, velver);
            k_force_gather<double, true><<<nblk(b.N, bs), bs, 0, st>>>(b);
        }
    } else if (newton3 == 5) {
        // registers capped for five 128-thread blocks per SM (20 warps); the
        // first evaluation (normals drawn) with the partners' records in an
        // async shared-memory ring, the second (normals read back from the
        // cache, far less arithmetic per pair) without: measured faster each
        if (precision == SDPD_PREC_SPLIT && velver == 1)
            k_force_fluid_lean<float, 5, 2><<<persistent_grid(k_force_fluid_lean<float, 5, 2>, LEAN_BLOCK, b.N),
                                              LEAN_BLOCK, 0, st>>>(b, velver);
        else if (precision == SDPD_PREC_SPLIT) {
            // velver 2: the pass that reads the cached normals, compiled
            // alone (two partner records per pair, the D record only for a
            // draw), then the drawing pass for the case where the cache is not
            // valid; each returns at once when the other one applies
            k_force_fluid_lean<float, 5, 0, 1>
                <<<persistent_grid(k_force_fluid_lean<float, 5, 0, 1>, LEAN_BLOCK, b.N), LEAN_BLOCK, 0, st>>>(b, velver);
            cudaMemsetAsync(b.work, 0, sizeof(unsigned long long), st);
            k_force_fluid_lean<float, 5, 0, 2>
                <<<persistent_grid(k_force_fluid_lean<float, 5, 0, 2>, LEAN_BLOCK, b.N), LEAN_BLOCK, 0, st>>>(b, velver);
        }
        else
            k_force_fluid<double><<<persistent_grid(k_force_fluid<double>, bs, b.N), bs, 0, st>>>(b, velver);
    } else if (b.tpp == 2 || b.tpp == 4) {
        // the direct pass with several lanes per particle: N x tpp threads
        const long long nt = b.N * (long long)b.tpp;
        if (precision == SDPD_PREC_SPLIT) {
            if (b.tpp == 2) k_force_fluid_tpp<float, 2><<<persistent_grid(k_force_fluid_tpp<float, 2>, bs, nt), bs, 0, st>>>(b, velver);
            else k_force_fluid_tpp<float, 4><<<persistent_grid(k_force_fluid_tpp<float, 4>, bs, nt), bs, 0, st>>>(b, velver);
        } else {
            if (b.tpp == 2) k_force_fluid_tpp<double, 2><<<persistent_grid(k_force_fluid_tpp<double, 2>, bs, nt), bs, 0, st>>>(b, velver);
            else k_force_fluid_tpp<double, 4><<<persistent_grid(k_force_fluid_tpp<double, 4>, bs, nt), bs, 0, st>>>(b, velver);
        }
    } else if (precision == SDPD_PREC_SPLIT && velver == 2) {
        // the pass reading the cached normals compiled alone (no D records,
        // no drawing code), then the drawing pass for an invalid cache; each
        // returns at once when the other one applies
        k_force_fluid<float, 1><<<persistent_grid(k_force_fluid<float, 1>, bs, b.N), bs, 0, st>>>(b, velver);
        cudaMemsetAsync(b.work, 0, sizeof(unsigned long long), st);
        k_force_fluid<float, 2><<<persistent_grid(k_force_fluid<float, 2>, bs, b.N), bs, 0, st>>>(b, velver);
    } else if (precision == SDPD_PREC_SPLIT) {
        k_force_fluid<float><<<persistent_grid(k_force_fluid<float>, bs, b.N), bs, 0, st>>>(b, velver);
    } else {
        k_force_fluid<double><<<persistent_grid(k_force_fluid<double>, bs, b.N), bs, 0, st>>>(b, velver);
    }
    if (b.nrigid) {
        const unsigned g = nblk(b.nrigid, RPB);
        const size_t smem = rigid_smem_bytes(b.cap);
        if (precision == SDPD_PREC_SPLIT) k_force_rigid<float><<<g, RB, smem, st>>>(b, velver);
        else k_force_rigid<double><<<g, RB, smem, st>>>(b, velver);
        if (velver == 2) k_hist_copy<<<nblk(b.nrigid, 64), 64, 0, st>>>(b);
    }
}

}  // namespace sdpd
