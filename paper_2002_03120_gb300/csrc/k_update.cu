// k_update.cu -- update(velver) of Algorithm 1 (velocity Verlet, boundary
// treatment, collision-method artificial viscosity) and the reductions of the
// viscometer read-out and the diagnostics.
#include "common.cuh"

namespace sdpd {

template <class R> struct VT;
template <> struct VT<float> { using T4 = float4; };
template <> struct VT<double> { using T4 = double4_32a; };

template <class R> __device__ __forceinline__ typename VT<R>::T4 *mirB(const Bufs &b);
template <> __device__ __forceinline__ float4 *mirB<float>(const Bufs &b) { return b.B32; }
template <> __device__ __forceinline__ double4_32a *mirB<double>(const Bufs &b) { return b.B64; }
template <class R> __device__ __forceinline__ typename VT<R>::T4 *mirC(const Bufs &b);
template <> __device__ __forceinline__ float4 *mirC<float>(const Bufs &b) { return b.C32; }
template <> __device__ __forceinline__ double4_32a *mirC<double>(const Bufs &b) { return b.C64; }

template <class R>
__device__ __forceinline__ void write_vel_mirror(const Bufs &b, long long s, const double *v, const double *w)
{
    auto *B = mirB<R>(b);
    auto *C = mirC<R>(b);
    auto Bs = B[s];
    auto Cs = C[s];
    Bs.x = (R)v[0]; Bs.y = (R)v[1]; Bs.z = (R)v[2];
    Cs.x = (R)w[0]; Cs.y = (R)w[1]; Cs.z = (R)w[2];
    B[s] = Bs;
    C[s] = Cs;
}

// a / d rounded to nearest from y = RN(1/d) by Markstein's method (P.
// Markstein, IBM J. Res. Dev. 34, 1990): q0 = RN(a y), the remainder
// r = a - d q0 is exact with a fused multiply-add, and RN(q0 + r y) is the
// correctly rounded quotient (no overflow or underflow here): the result of
// the division a / d, with one multiply and two multiply-adds.
__device__ __forceinline__ double div_rn(double a, double d, double y)
{
    const double q0 = __dmul_rn(a, y);
    const double r = __fma_rn(-q0, d, a);
    return __fma_rn(r, y, q0);
}

// Comparisons on the integer pipe (the FP64 pipe of this part runs at 1/64 of
// the FP32 rate and bounds the update): key(x) orders like x for every
// non-NaN double, -0 and +0 alike; a NaN takes a branch the IEEE comparison
// would not, but stays NaN and is flagged either way.
__device__ __forceinline__ long long ord_key(double x)
{
    const long long k = __double_as_longlong(x);
    return k >= 0 ? k : (long long)(0x8000000000000000ull - (unsigned long long)k);
}
__device__ __forceinline__ bool finite_bits(double x)
{
    return ((unsigned long long)__double_as_longlong(x) & 0x7FF0000000000000ull) != 0x7FF0000000000000ull;
}

// Velocity Verlet (Eqs. newton1, newton2): v += dt/2 F/m, w += dt/2 N/I;
// velver 1 also drifts x += dt v, wraps periodic axes and mirrors particles
// that crossed a wall plane (normal velocity reversed).  The arithmetic is
// written without fused multiply-adds so it repeats the oracle bit for bit;
// the decisions (wrap, reflection, periodic jump, finiteness) are taken on
// the integer pipe from the bit patterns, with the oracle's outcomes.
template <class R>
__global__ void k_integrate(Bufs b, int velver)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (velver == 1 && s == 0) *b.aclose_ok = 0;   // the drift moves the particles
    if (s >= b.N) return;
    const int g = b.perm[s];
    const int t = b.type[g];
    if (t != T_FLUID && t != T_RIGID) return;
    const Inst &I = b.inst[b.pinst[g]];
    const double im = b.m[g], iI = b.Iner[g], rm = b.rm[g], rI = b.rI[g];
    const double hdt = I.hdt;
    double v[3], w[3], x[3];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        v[a] = __dadd_rn(b.v[3 * g + a], __dmul_rn(hdt, div_rn(b.F[3 * g + a], im, rm)));
        w[a] = __dadd_rn(b.w[3 * g + a], __dmul_rn(hdt, div_rn(b.T[3 * g + a], iI, rI)));
    }
    if (velver == 1) {
        const double dt = I.dt;
        double dl[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double x0 = b.x[3 * g + a];
            double xa = __dadd_rn(x0, __dmul_rn(dt, v[a]));
            const double lo = I.origin[a], hi = I.dom_hi[a], L = I.box[a];
            const long long kx = ord_key(xa);
            const bool per = I.periodic[a];
            if (per) {
                if (kx < ord_key(lo)) xa = __dadd_rn(xa, L);
                else if (kx >= ord_key(hi)) xa = __dsub_rn(xa, L);
            } else {
                if (kx < ord_key(lo)) { xa = __dadd_rn(lo, __dsub_rn(lo, xa)); v[a] = -v[a]; }
                else if (kx > ord_key(hi)) { xa = __dsub_rn(hi, __dsub_rn(xa, hi)); v[a] = -v[a]; }
            }
            x[a] = xa;
            b.x[3 * g + a] = xa;
            ok &= finite_bits(xa);
            // displacement without the periodic jump (|d| > L/2 decided on the bits)
            double d = __dsub_rn(xa, x0);
            if (per && abs_bits(d) > I.hbox_bits[a]) d = (__double_as_longlong(d) > 0) ? __dsub_rn(d, L) : __dadd_rn(d, L);
            dl[a] = d;
        }
        // keep the mirrors of the unchanged slot order current: cell-relative
        // coordinates move by the displacement (the build cell stays), the
        // displacement since the build decides whether the list still holds
        double4_32a xl = b.xl64[s], ds = b.dsp[s];
        xl.x += dl[0]; xl.y += dl[1]; xl.z += dl[2];
        ds.x += dl[0]; ds.y += dl[1]; ds.z += dl[2];
        b.xl64[s] = xl;
        b.dsp[s] = ds;
        float4 a32 = b.A32[s];
        a32.x = (float)xl.x; a32.y = (float)xl.y; a32.z = (float)xl.z;
        b.A32[s] = a32;
        if (b.A64) {
            double4_32a a64 = b.A64[s];
            a64.x = x[0]; a64.y = x[1]; a64.z = x[2];
            b.A64[s] = a64;
        }
        if (fma(ds.z, ds.z, fma(ds.y, ds.y, ds.x * ds.x)) > I.half_skin * I.half_skin) *b.need_build = 1;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        b.v[3 * g + a] = v[a];
        b.w[3 * g + a] = w[a];
        ok &= finite_bits(v[a]) & finite_bits(w[a]);
    }
    if (!ok) atomicOr(b.err, ERR_NONFINITE);
    write_vel_mirror<R>(b, s, v, w);
}

// Absorb uploaded state (sdpd_upload_state) into a context whose lists are
// valid: each particle moves by its displacement (minimum image on periodic
// axes), the cell-relative mirrors and the displacement since the build move
// with it, and the velocity mirrors take the uploaded velocities.  A
// displacement beyond half the skin requests a rebuild (the gated build of
// the next step), exactly as after a drift; otherwise the lists still hold
// every pair within h.
template <class R>
__global__ void k_absorb(Bufs b, const double *__restrict__ xs, int has_x)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.N) return;
    const int g = b.perm[s];
    const Inst &I = b.inst[b.pinst[g]];
    if (has_x) {
        double dl[3], x[3];
        for (int a = 0; a < 3; ++a) {
            const double x0 = b.x[3 * g + a], xa = xs[3 * g + a];
            double d = xa - x0;
            if (I.periodic[a]) {
                if (d > 0.5 * I.box[a]) d -= I.box[a];
                else if (d < -0.5 * I.box[a]) d += I.box[a];
            }
            dl[a] = d;
            x[a] = xa;
            b.x[3 * g + a] = xa;
        }
        double4_32a xl = b.xl64[s], ds = b.dsp[s];
        xl.x += dl[0]; xl.y += dl[1]; xl.z += dl[2];
        ds.x += dl[0]; ds.y += dl[1]; ds.z += dl[2];
        b.xl64[s] = xl;
        b.dsp[s] = ds;
        float4 a32 = b.A32[s];
        a32.x = (float)xl.x; a32.y = (float)xl.y; a32.z = (float)xl.z;
        b.A32[s] = a32;
        if (b.A64) {
            double4_32a a64 = b.A64[s];
            a64.x = x[0]; a64.y = x[1]; a64.z = x[2];
            b.A64[s] = a64;
        }
        if (ds.x * ds.x + ds.y * ds.y + ds.z * ds.z > I.half_skin * I.half_skin) *b.need_build = 1;
    }
    const double v[3] = { b.v[3 * g], b.v[3 * g + 1], b.v[3 * g + 2] };
    const double w[3] = { b.w[3 * g], b.w[3 * g + 1], b.w[3 * g + 2] };
    write_vel_mirror<R>(b, s, v, w);
    if (s == 0) *b.aclose_ok = 0;   // positions changed
}

// Collision-method artificial viscosity: pairs of mobile particles closer
// than artvis_alpha dx that approach exchange momentum as an inelastic
// collision with restitution artvis_e; Jacobi form (pre-correction
// velocities), momentum-conserving.
__global__ void k_artvis(Bufs b)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.N) return;
    const int g = b.perm[s];
    const int t = b.type[g];
    double dv[3] = { 0.0, 0.0, 0.0 };
    const Inst &I = b.inst[b.pinst[g]];
    // the density pass of these positions marked the particles that have a
    // mobile neighbour inside the collision radius; the others skip the scan
    const bool marked = !*b.aclose_ok || b.aclose[s];
    if ((t == T_FLUID || t == T_RIGID) && I.artvis && marked) {
        const double xi[3] = { b.x[3 * g], b.x[3 * g + 1], b.x[3 * g + 2] };
        const double vi[3] = { b.v[3 * g], b.v[3 * g + 1], b.v[3 * g + 2] };
        const double mi = b.m[g];
        const int n = b.ncnt[s];
        const Geo<float> geo(I);
        const float4 Ai = b.A32[s];
        const float r2hi = I.artvis_r2f_hi;
        for (int k = 0; k < n; ++k) {
            const uint32_t e = (uint32_t)b.nbr[(long long)k * b.Npad + s];
            if (e & NB_FAR) continue;
            // float prefilter on the cell-relative mirror; exact test below
            const float4 Aj = b.A32[e];
            float fx, fy, fz;
            geo.disp(Ai, Aj, fx, fy, fz);
            if (fx * fx + fy * fy + fz * fz > r2hi) continue;
            const int gj = b.perm[e];
            const int tj = b.type[gj];
            if (tj != T_FLUID && tj != T_RIGID) continue;
            double r[3];
            for (int a = 0; a < 3; ++a) {
                double d = xi[a] - b.x[3 * gj + a];
                if (I.periodic[a]) {
                    if (d > 0.5 * I.box[a]) d -= I.box[a];
                    else if (d < -0.5 * I.box[a]) d += I.box[a];
                }
                r[a] = d;
            }
            const double rr = sqrt((r[0] * r[0] + r[1] * r[1]) + r[2] * r[2]);
            if (!(rr < I.artvis_rlim)) continue;
            const double e3[3] = { r[0] / rr, r[1] / rr, r[2] / rr };
            const double ve = (vi[0] - b.v[3 * gj]) * e3[0] + (vi[1] - b.v[3 * gj + 1]) * e3[1] +
                              (vi[2] - b.v[3 * gj + 2]) * e3[2];
            if (!(ve < 0.0)) continue;
            const double mj = b.m[gj];
            const double c = -(1.0 + I.artvis_e) * mj / (mi + mj) * ve;
            for (int a = 0; a < 3; ++a) dv[a] += c * e3[a];
        }
    }
    b.dv[3 * g] = dv[0];
    b.dv[3 * g + 1] = dv[1];
    b.dv[3 * g + 2] = dv[2];
}

template <class R>
__global__ void k_artvis_apply(Bufs b)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.N) return;
    const int g = b.perm[s];
    const int t = b.type[g];
    if (t != T_FLUID && t != T_RIGID) return;
    double v[3], w[3];
    for (int a = 0; a < 3; ++a) {
        v[a] = b.v[3 * g + a] + b.dv[3 * g + a];
        b.v[3 * g + a] = v[a];
        w[a] = b.w[3 * g + a];
    }
    write_vel_mirror<R>(b, s, v, w);
}

__global__ void k_step_done(Bufs b)
{
    *b.step += 1;
    *b.fresh = 0;
}

// ----------------------------------------------------- viscometer read-out
// probe layout: [0, nb) velocity sums, [nb, 2nb) counts, [2nb, 2nb+4)
// signed velocity sums and counts of the two halves.
__global__ void k_probe(Bufs b, int inst, int nb)
{
    const Inst &I = b.inst[inst];
    const long long g = I.p_begin + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= I.p_end) return;
    if (b.type[g] != T_FLUID) return;
    const int ax = I.split_axis, fa = I.body_axis;
    const double rel = b.x[3 * g + ax] - I.origin[ax];
    int bin = (int)floor(rel / I.box[ax] * nb);
    bin = bin < 0 ? 0 : (bin >= nb ? nb - 1 : bin);
    const double u = b.v[3 * g + fa];
    atomicAdd(&b.probe[bin], u);
    atomicAdd(&b.probe[nb + bin], 1.0);
    const int half = (rel < 0.5 * I.box[ax]) ? 0 : 1;
    atomicAdd(&b.probe[2 * nb + half], half == 0 ? u : -u);
    atomicAdd(&b.probe[2 * nb + 2 + half], 1.0);
    atomicAdd(&b.probe[2 * nb + 4 + bin], rel);   // mean position of the slab's particles
}

// diagnostics layout in probe: [0..2] momentum, [3] sum m v^2, [4] sum m,
// [5] count mobile, [6] max |v| (as ordered bits), [7] min d, [8] max d,
// [9] non-finite count
__global__ void k_diag(Bufs b, int inst)
{
    const Inst &I = b.inst[inst];
    const long long g = I.p_begin + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= I.p_end) return;
    const int t = b.type[g];
    double nonf = 0.0;
    for (int a = 0; a < 3; ++a)
        nonf += (!isfinite(b.x[3 * g + a])) + (!isfinite(b.v[3 * g + a])) + (!isfinite(b.w[3 * g + a]));
    if (nonf > 0) atomicAdd(&b.probe[9], nonf);
    const long long s = b.slot_of[g];
    if (t != T_OUTER) {
        const double d = b.sd[s];
        atomicMin((unsigned long long *)&b.probe[7], (unsigned long long)__double_as_longlong(d));
        atomicMax((unsigned long long *)&b.probe[8], (unsigned long long)__double_as_longlong(d));
    }
    if (t != T_FLUID && t != T_RIGID) return;
    const double m = b.m[g];
    const double v0 = b.v[3 * g], v1 = b.v[3 * g + 1], v2 = b.v[3 * g + 2];
    atomicAdd(&b.probe[0], m * v0);
    atomicAdd(&b.probe[1], m * v1);
    atomicAdd(&b.probe[2], m * v2);
    const double v2s = v0 * v0 + v1 * v1 + v2 * v2;
    atomicAdd(&b.probe[3], m * v2s);
    atomicAdd(&b.probe[4], m);
    atomicAdd(&b.probe[5], 1.0);
    atomicMax((unsigned long long *)&b.probe[6], (unsigned long long)__double_as_longlong(sqrt(v2s)));
}

// Unordered pairs within h evaluated by the force pass (>= 1 mobile member).
__global__ void k_count_pairs(Bufs b)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c = 0;
    if (s < b.N) {
        const int ti = b.stype[s];
        if (ti == T_FLUID || ti == T_RIGID) {
            const int n = b.ncnt[s];
            const int gi = b.perm[s];
            const Inst &I = b.inst[b.pinst[gi]];
            for (int k = 0; k < n; ++k) {
                const uint32_t e = (uint32_t)b.nbr[(long long)k * b.Npad + s];
                if (e & NB_FAR) continue;
                if (!exact_within(b, I, gi, b.perm[e])) continue;
                const int tj = b.stype[e];
                const bool mj = (tj == T_FLUID || tj == T_RIGID);
                c += mj ? ((long long)e > s ? 1u : 0u) : 1u;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(b.pair_count, c);
}

// Flags of the list entries within h at the current positions (exact test).
__global__ void k_mark_pairs(Bufs b, uint8_t *flags)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.N) return;
    const int gi = b.perm[s];
    const Inst &I = b.inst[b.pinst[gi]];
    const int n = b.ncnt[s];
    for (int k = 0; k < n; ++k) {
        const uint32_t e = (uint32_t)b.nbr[(long long)k * b.Npad + s];
        flags[(long long)k * b.Npad + s] =
            (!(e & NB_FAR) && exact_within(b, I, gi, b.perm[e & ~NB_FAR])) ? 1 : 0;
    }
}

// ---------------------------------------------------------------- launchers
static inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

void launch_integrate(const Bufs &b, int precision, int velver, int any_artvis, cudaStream_t st)
{
    if (!b.N) return;
    if (precision == SDPD_PREC_SPLIT) k_integrate<float><<<nblk(b.N, 256), 256, 0, st>>>(b, velver);
    else k_integrate<double><<<nblk(b.N, 256), 256, 0, st>>>(b, velver);
    if (velver == 2 && any_artvis) {
        k_artvis<<<nblk(b.N, 128), 128, 0, st>>>(b);
        if (precision == SDPD_PREC_SPLIT) k_artvis_apply<float><<<nblk(b.N, 256), 256, 0, st>>>(b);
        else k_artvis_apply<double><<<nblk(b.N, 256), 256, 0, st>>>(b);
    }
}

void launch_step_done(const Bufs &b, cudaStream_t st) { k_step_done<<<1, 1, 0, st>>>(b); }

void launch_probe(const Bufs &b, int inst, int nbins, cudaStream_t st, long long n)
{
    cudaMemsetAsync(b.probe, 0, sizeof(double) * (3 * nbins + 4), st);
    if (n) k_probe<<<nblk(n, 256), 256, 0, st>>>(b, inst, nbins);
}

void launch_diag(const Bufs &b, int inst, cudaStream_t st, long long n)
{
    cudaMemsetAsync(b.probe, 0, sizeof(double) * 16, st);
    // min d starts at +inf bits
    const double big = 1e308;
    cudaMemcpyAsync(&b.probe[7], &big, sizeof(double), cudaMemcpyHostToDevice, st);
    if (n) k_diag<<<nblk(n, 256), 256, 0, st>>>(b, inst);
}

void launch_mark_pairs(const Bufs &b, uint8_t *flags, cudaStream_t st)
{
    if (b.N) k_mark_pairs<<<nblk(b.N, 128), 128, 0, st>>>(b, flags);
}

// The six normals of the random term (Eq. FijT) of given pairs, as the pair
// kernels draw them.
template <class R>
__global__ void k_noise_normals(long long n, const uint32_t *gi, const uint32_t *gj, uint32_t step, uint32_t k0,
                                uint32_t k1, double *out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    R z[6];
    pair_normals<R>(gi[i], gj[i], step, k0, k1, z[0], z[1], z[2], z[3], z[4], z[5]);
#pragma unroll
    for (int k = 0; k < 6; ++k) out[6 * i + k] = (double)z[k];
}

// Raw Philox4x32-10 blocks for given counters and keys (the generator of
// the random term, exposed so its bits can be checked against published
// known-answer vectors).
__global__ void k_philox_raw(long long n, const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint4 r = philox4x32_10(c, key[2 * i], key[2 * i + 1]);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

void launch_philox_raw(long long n, const uint32_t *ctr, const uint32_t *key, uint32_t *out, cudaStream_t st)
{
    if (n) k_philox_raw<<<nblk(n, 256), 256, 0, st>>>(n, ctr, key, out);
}

void launch_noise_normals(int precision, long long n, const uint32_t *gi, const uint32_t *gj, uint32_t step,
                          uint32_t k0, uint32_t k1, double *out, cudaStream_t st)
{
    if (!n) return;
    if (precision == SDPD_PREC_FP64)
        k_noise_normals<double><<<nblk(n, 256), 256, 0, st>>>(n, gi, gj, step, k0, k1, out);
    else
        k_noise_normals<float><<<nblk(n, 256), 256, 0, st>>>(n, gi, gj, step, k0, k1, out);
}

void launch_absorb(const Bufs &b, int precision, const double *xs, int has_x, cudaStream_t st)
{
    if (!b.N) return;
    if (precision == SDPD_PREC_SPLIT) k_absorb<float><<<nblk(b.N, 256), 256, 0, st>>>(b, xs, has_x);
    else k_absorb<double><<<nblk(b.N, 256), 256, 0, st>>>(b, xs, has_x);
}

void launch_count_pairs(const Bufs &b, cudaStream_t st)
{
    cudaMemsetAsync(b.pair_count, 0, sizeof(unsigned long long), st);
    if (b.N) k_count_pairs<<<nblk(b.N, 256), 256, 0, st>>>(b);
}

}  // namespace sdpd
