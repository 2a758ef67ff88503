// k_cells.cu -- compute_neighbor_list (Algorithm 1, Section 3.2) on the GPU.
//
// The paper's background grid with linked lists is replaced by a counting
// sort of the particles into Morton-ranked cells:
//   K1 cell key per particle + atomic per-cell count      (HBM bound, 1 pass)
//   K2 exclusive scan of the counts -> cell starts
//   K3 scatter into cell ranges, K4 rank by gid inside each cell (deterministic
//      order, so every later sum is reproducible bit for bit)
//   K5 gather of the cell-sorted mirrors (float4 / double4 records)
//   K6 per particle, the list of neighbours j != i within the build
//      radius rb = h (1 + skin) from the surrounding cells
//   K7 reverse index of the Newton-3 force pass
// The list is a superset of the pairs within h; every consumer re-decides
// r_ij < h exactly, so the evaluated pair set equals the paper's.  The list
// stays valid while no particle has moved more than skin h / 2 since the
// build; the drift raises `need_build` when one has, and every kernel here
// is gated on that flag inside the captured step.
#include "common.cuh"

namespace sdpd {

#define GATE                                                                                    \
    if (gate && *gate == 0) return;

__device__ __forceinline__ int cell_coord(double x, double lo, double inv_cs, int nc, bool &out, bool &nonfinite)
{
    const double f = floor((x - lo) * inv_cs);
    nonfinite = !(fabs(f) < 1e9);   // NaN or a runaway coordinate
    const int k = nonfinite ? 0 : (int)f;
    out = (k < 0) || (k >= nc);
    return k < 0 ? 0 : (k >= nc ? nc - 1 : k);
}

__global__ void k_cell_clear(Bufs b, const int *gate)
{
    GATE;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < b.ncell_total) b.ccount[c] = 0;
}

__global__ void k_cell_keys(Bufs b, const int *gate)
{
    GATE;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= b.N) return;
    const Inst &I = b.inst[b.pinst[g]];
    int c[3];
    bool bad = false, nf = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        bool o, f;
        c[a] = cell_coord(b.x[3 * g + a], I.lo[a], I.inv_cs[a], I.nc[a], o, f);
        bad |= o;
        nf |= f;
    }
    if (nf) atomicOr(b.err, ERR_NONFINITE);
    else if (bad) atomicOr(b.err, ERR_DOMAIN);
    const int lin = (c[2] * I.nc[1] + c[1]) * I.nc[0] + c[0];
    const int key = I.cell_base + b.cell_rank[I.cell_base + lin];
    b.key[g] = key;
    b.slot_in_cell[g] = atomicAdd(&b.ccount[key], 1);
}

// --- exclusive scan of the cell counts (three phases, 1024 cells per block)
__device__ __forceinline__ int warp_incl_scan(int v)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) >= o) v += t;
    }
    return v;
}

__device__ int block_excl_scan(int v, int *total)
{
    __shared__ int ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) ws[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int s = (lane < (int)(blockDim.x >> 5)) ? ws[lane] : 0;
        s = warp_incl_scan(s);
        ws[lane] = s;
    }
    __syncthreads();
    const int off = wid ? ws[wid - 1] : 0;
    *total = ws[(blockDim.x >> 5) - 1];
    __syncthreads();
    return off + inc - v;
}

__global__ void k_scan_local(Bufs b, const int *gate)
{
    GATE;
    const int n = b.ncell_total;
    const int i = blockIdx.x * 1024 + threadIdx.x;
    const int v = i < n ? b.ccount[i] : 0;
    int tot;
    const int e = block_excl_scan(v, &tot);
    if (i < n) b.cstart[i] = e;
    if (threadIdx.x == 0) b.scan_partials[blockIdx.x] = tot;
}

__global__ void k_scan_partials(Bufs b, int nblk, const int *gate)
{
    GATE;
    // one block of 1024 threads, sequential over chunks
    int carry = 0;
    for (int base = 0; base < nblk; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < nblk ? b.scan_partials[i] : 0;
        int tot;
        const int e = block_excl_scan(v, &tot);
        if (i < nblk) b.scan_partials[i] = carry + e;
        carry += tot;
        __syncthreads();
    }
}

__global__ void k_scan_add(Bufs b, const int *gate)
{
    GATE;
    const int n = b.ncell_total;
    const int i = blockIdx.x * 1024 + threadIdx.x;
    if (i < n) b.cstart[i] += b.scan_partials[blockIdx.x];
    if (i == 0) b.cstart[n] = (int)b.N;
}

__global__ void k_scatter(Bufs b, const int *gate)
{
    GATE;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= b.N) return;
    b.tmp_perm[b.cstart[b.key[g]] + b.slot_in_cell[g]] = (int)g;
}

// Rank of each particle among its cell's members by gid (stable, unique).
__global__ void k_rank(Bufs b, const int *gate)
{
    GATE;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= b.N) return;
    const int g = b.tmp_perm[t];
    const int c = b.key[g];
    const int s0 = b.cstart[c], s1 = b.cstart[c + 1];
    int r = 0;
    for (int u = s0; u < s1; ++u) r += (b.tmp_perm[u] < g);
    b.perm[s0 + r] = g;
    b.slot_of[g] = s0 + r;
}

// Cell-sorted mirrors for the pair kernels; resets the displacement since
// the build.
__global__ void k_gather(Bufs b, int precision, const int *gate)
{
    GATE;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.N) return;
    const int g = b.perm[s];
    const int ii = b.pinst[g];
    const Inst &I = b.inst[ii];
    const int t = b.type[g];
    b.stype[s] = t;
    const double x0 = b.x[3 * g], x1 = b.x[3 * g + 1], x2 = b.x[3 * g + 2];
    const uint32_t lg = (uint32_t)(g - I.p_begin);
    {
        // cell-relative coordinates (both precisions: the neighbour search
        // and the split-precision pair kernels work on them)
        int c[3];
        double xl[3];
        const double xs[3] = { x0, x1, x2 };
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            bool o, f;
            c[a] = cell_coord(xs[a], I.lo[a], I.inv_cs[a], I.nc[a], o, f);
            xl[a] = xs[a] - (I.lo[a] + (double)c[a] * I.cs[a]);
        }
        b.A32[s] = make_float4((float)xl[0], (float)xl[1], (float)xl[2],
                               __uint_as_float(pack_cell(t, c[0], c[1], c[2])));
        b.skey[s] = b.key[g];
        b.xl64[s] = make_double4_32a(xl[0], xl[1], xl[2], 0.0);
        b.dsp[s] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    }
    if (precision == SDPD_PREC_SPLIT) {
        b.B32[s] = make_float4((float)b.v[3 * g], (float)b.v[3 * g + 1], (float)b.v[3 * g + 2],
                               (float)b.R[g]);
        b.C32[s] = make_float4((float)b.w[3 * g], (float)b.w[3 * g + 1], (float)b.w[3 * g + 2],
                               (float)b.m[g]);
        b.D32[s].w = __uint_as_float(lg);
    } else {
        b.A64[s] = make_double4_32a(x0, x1, x2, (double)t);
        b.B64[s] = make_double4_32a(b.v[3 * g], b.v[3 * g + 1], b.v[3 * g + 2], b.R[g]);
        b.C64[s] = make_double4_32a(b.w[3 * g], b.w[3 * g + 1], b.w[3 * g + 2], b.m[g]);
        b.D64[s].w = (double)lg;
    }
}

// Neighbour list of particle (slot) s: candidates from the cells around s's
// cell (cells are at least max(rb, largest sphere diameter + skin) wide,
// periodic axes at least 3 cells).  A pair is listed when r < rb (float test:
// the list only has to be a superset of the pairs within h), or when both are
// rigid and r < R_i + R_j + skin h (contact range; flagged NB_FAR).
//
// Newton-3 ownership, balanced so that every particle owns about half of its
// pairs whatever its position in the cell: the pair of instance-local slots
// a < b belongs to a when bit 15 of the hash (a * 0x9E3779B1) ^
// (b * 0x85EBCA77) is set, else to b.  The list is written as [owned][not
// owned], the owned part ascending in slot (cells visited in ascending key),
// the other descending, so the owned pairs are the prefix [0, nfirst) and a
// partner's position is found by binary search in it.
__device__ __forceinline__ bool pair_owned(long long s, int j, int base)
{
    // instance-local slots: an instance owns the same pairs alone or batched
    const uint32_t lo = (uint32_t)(min((long long)j, s) - base), hi = (uint32_t)(max((long long)j, s) - base);
    const uint32_t h = (lo * 0x9E3779B1u) ^ (hi * 0x85EBCA77u);
    const bool low_owns = (h >> 15) & 1u;
    return low_owns == (s < j);
}


// The candidate test of a pair (i, j) with j's record Aj and the offset
// (sx, sy, sz) of j's cell: within rb (float), or both rigid and within
// contact range (flagged NB_FAR).
__device__ __forceinline__ bool nb_test(const Bufs &b, const Inst &I, const float4 &Ai, int ti, float Ri,
                                        int j, const float4 &Aj, float sx, float sy, float sz, uint32_t &entry,
                                        int &tj)
{
    tj = unpack_type(__float_as_uint(Aj.w));
    const float dx = (Ai.x - Aj.x) - sx, dy = (Ai.y - Aj.y) - sy, dz = (Ai.z - Aj.z) - sz;
    const float r2f = dx * dx + dy * dy + dz * dz;
    entry = (uint32_t)j;
    if (r2f < I.rb2f) return true;
    if (ti == T_RIGID && tj == T_RIGID) {
        const float lim = (Ri + (float)b.R[b.perm[j]] + (float)(2.0 * I.half_skin)) * 1.0001f;
        entry |= NB_FAR;
        return r2f < lim * lim;
    }
    return false;
}

// One warp per cell, its particles 32 at a time: all lanes share the cell's
// 27 neighbour cells, so the candidates' records are read once per warp --
// 32 consecutive records, coalesced, into shared memory -- and every lane
// tests them from there (broadcast reads) instead of each lane loading every
// candidate from global memory.  Cells and candidates are visited in
// ascending order, as a per-particle scan would.
constexpr int NB_WARPS = 8;

__global__ void __launch_bounds__(NB_WARPS * 32) k_neighbors(Bufs b, const int *gate)
{
    GATE;
    __shared__ float4 stage[NB_WARPS][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * NB_WARPS + w;
    if (c >= b.ncell_total) return;   // the whole warp
    const int s0 = b.cstart[c], s1 = b.cstart[c + 1];
    if (s0 == s1) return;
    const int *adj = b.cell_adj + (long long)c * 27;
    const Inst &I = b.inst[b.pinst[b.perm[s0]]];   // a cell belongs to one instance
    const int base = b.cstart[I.cell_base];           // first slot of the instance
    const long long Np = b.Npad;
    const int cap = b.cap;
    for (int chunk = s0; chunk < s1; chunk += 32) {
        const int s = chunk + lane;
        const bool act = s < s1;
        int ti = T_FLUID;
        float Ri = 0.f;
        float4 Ai = make_float4(0.f, 0.f, 0.f, 0.f);
        if (act) {
            ti = b.stype[s];
            Ri = (ti == T_RIGID) ? (float)b.R[b.perm[s]] : 0.f;
            Ai = b.A32[s];
        }
        int *col = b.nbr + s;   // this particle's column, entry k at col[k * Np]
        // one scan in ascending slot order: owned pairs from the front, the
        // others from the back of the column (so in descending positions)
        int nf = 0, m = 0;
        bool rig = false;
        for (int q = 0; q < 27; ++q) {
            const int code = adj[q];
            if (code < 0) break;
            const int key = code >> 5, oc = code & 31;
            const float sx = (float)(oc % 3 - 1) * I.csf[0], sy = (float)((oc / 3) % 3 - 1) * I.csf[1],
                        sz = (float)(oc / 9 - 1) * I.csf[2];
            const int j0 = b.cstart[key], j1 = b.cstart[key + 1];
            for (int jb = j0; jb < j1; jb += 32) {
                const int jj = jb + lane;
                __syncwarp();
                stage[w][lane] = jj < j1 ? b.A32[jj] : make_float4(0.f, 0.f, 0.f, 0.f);
                __syncwarp();
                if (!act) continue;
                const int cnt = min(32, j1 - jb);
                for (int t = 0; t < cnt; ++t) {
                    const int j = jb + t;
                    uint32_t entry;
                    int tj;
                    if (j == s || !nb_test(b, I, Ai, ti, Ri, j, stage[w][t], sx, sy, sz, entry, tj)) continue;
                    rig |= (tj == T_RIGID);
                    if (pair_owned(s, j, base)) {
                        if (nf + m < cap) col[(long long)nf * Np] = (int)entry;
                        ++nf;
                    } else {
                        if (nf + m < cap) col[(long long)(cap - 1 - m) * Np] = (int)entry;
                        ++m;
                    }
                }
            }
        }
        if (!act) continue;
        const int n = nf + m;
        // the pair buffer holds capown rows of owned and of non-owned entries
        if (nf > b.capown || m > b.capown) atomicOr(b.err, ERR_PAIR_CAP);
        if (n > cap) {
            atomicOr(b.err, ERR_NBR_CAP);
        } else {
            // the back region [cap - m, cap) holds the non-owned entries in
            // descending slot order: move it down to [nf, n) as it is
            // (destination below the source, so an ascending copy never
            // overwrites an entry still to be read); only the owned prefix
            // needs ascending order (the reverse index searches it)
            if (nf < cap - m)
                for (int k = 0; k < m; ++k) col[(long long)(nf + k) * Np] = col[(long long)(cap - m + k) * Np];
        }
        b.nfirst[s] = min(nf, min(cap, b.capown));
        b.ncnt[s] = min(n, cap);
        b.nbflag[s] = rig ? 1 : 0;
    }
}

// For every non-owned entry k of s (positions [nfirst, n)), the position r
// of s in the partner j's owned prefix (ascending), by binary search; four
// searches run interleaved so their loads overlap.  Both directions are kept,
// in disjoint rows of rev: rev[k][s] = r (where s reads j's result in j's
// column) and rev[r][j] = k - nfirst(s) (where j writes its result in s's
// column); each owned entry of j gets exactly one.
__device__ __forceinline__ int nb_at(const Bufs &b, int i, int k)
{
    return (int)((uint32_t)__ldg(b.nbr + (long long)k * b.Npad + i) & ~NB_FAR);
}

__global__ void k_rev(Bufs b, const int *gate)
{
    GATE;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.N) return;
    const long long Np = b.Npad;
    const int first = b.nfirst[s], n = b.ncnt[s];
    constexpr int G = 4;  // (owned prefixes are <= capown, checked at the build)
    for (int k0 = first; k0 < n; k0 += G) {
        int part[G], lo[G], hi[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int k = k0 + g;
            part[g] = k < n ? (int)((uint32_t)b.nbr[(long long)k * Np + s] & ~NB_FAR) : -1;
            lo[g] = 0;
            hi[g] = part[g] >= 0 ? b.nfirst[part[g]] : 0;
        }
        int end[G];
#pragma unroll
        for (int g = 0; g < G; ++g) end[g] = hi[g];
        bool active = true;
        while (active) {
            active = false;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (lo[g] < hi[g]) {
                    const int mid = (lo[g] + hi[g]) >> 1;
                    if (nb_at(b, part[g], mid) < (int)s) lo[g] = mid + 1;
                    else hi[g] = mid;
                    active = true;
                }
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int k = k0 + g;
            if (k >= n) break;
            const bool ok = lo[g] < end[g] && nb_at(b, part[g], lo[g]) == (int)s;
            if (!ok || k - first >= b.capown) atomicOr(b.err, ERR_REV);
            b.rev[(long long)k * Np + s] = (uint16_t)(ok ? lo[g] : 0);
            if (ok && k - first < b.capown) b.rev[(long long)lo[g] * Np + part[g]] = (uint16_t)(k - first);
        }
    }
}

// Closes the build: a new list epoch, the gate shut until the skin is used up.
__global__ void k_build_done(Bufs b, const int *gate)
{
    GATE;
    *b.list_epoch += 1u;
    *b.need_build = 0;
    *b.fresh = 1;
    *b.aclose_ok = 0;   // slots were reassigned
}

// ---------------------------------------------------------------- launchers
static inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

void launch_build(const Bufs &b, int precision, int need_rev, const int *gate, cudaStream_t st)
{
    const int nc = b.ncell_total;
    const int nbk = (nc + 1023) / 1024;
    k_cell_clear<<<nblk(nc, 256), 256, 0, st>>>(b, gate);
    if (b.N) k_cell_keys<<<nblk(b.N, 256), 256, 0, st>>>(b, gate);
    k_scan_local<<<nbk, 1024, 0, st>>>(b, gate);
    k_scan_partials<<<1, 1024, 0, st>>>(b, nbk, gate);
    k_scan_add<<<nbk, 1024, 0, st>>>(b, gate);
    if (b.N) {
        k_scatter<<<nblk(b.N, 256), 256, 0, st>>>(b, gate);
        k_rank<<<nblk(b.N, 256), 256, 0, st>>>(b, gate);
        k_gather<<<nblk(b.N, 256), 256, 0, st>>>(b, precision, gate);
        k_neighbors<<<nblk(nc, NB_WARPS), NB_WARPS * 32, 0, st>>>(b, gate);
        if (need_rev) k_rev<<<nblk(b.N, 128), 128, 0, st>>>(b, gate);
    }
    k_build_done<<<1, 1, 0, st>>>(b, gate);
}

}  // namespace sdpd
