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
#include <algorithm>

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
// cell (cells are at least max(rb, largest sphere diameter + skin) / sub
// wide and the stencil reaches sub cells each way, sub = 1 or 2; periodic
// axes at least 2 sub + 1 cells).  A pair is listed when r < rb (float test:
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
// neighbour cells (27, or 125 with half-size cells), so the candidates' records are read once per warp --
// 32 consecutive records, coalesced, into shared memory -- and every lane
// tests them from there (broadcast reads) instead of each lane loading every
// candidate from global memory.  Cells and candidates are visited in
// ascending order, as a per-particle scan would.
constexpr int NB_WARPS = 8;

// The lists of cell c's particles [s0, s1), one lane per particle; stage:
// 32 float4 of this warp's shared memory.
__device__ void nb_scan_cell(const Bufs &b, int c, int s0, int s1, float4 *stage, int lane)
{
    const int *adj = b.cell_adj + (long long)c * ADJ;
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
        for (int q = 0; q < ADJ; ++q) {
            const int code = adj[q];
            if (code < 0) break;
            const int key = code >> 7, oc = code & 127;
            const float sx = (float)(oc % 5 - 2) * I.csf[0], sy = (float)((oc / 5) % 5 - 2) * I.csf[1],
                        sz = (float)(oc / 25 - 2) * I.csf[2];
            const int j0 = b.cstart[key], j1 = b.cstart[key + 1];
            for (int jb = j0; jb < j1; jb += 32) {
                const int jj = jb + lane;
                __syncwarp();
                stage[lane] = jj < j1 ? b.A32[jj] : make_float4(0.f, 0.f, 0.f, 0.f);
                __syncwarp();
                if (!act) continue;
                const int cnt = min(32, j1 - jb);
                for (int t = 0; t < cnt; ++t) {
                    const int j = jb + t;
                    uint32_t entry;
                    int tj;
                    if (j == s || !nb_test(b, I, Ai, ti, Ri, j, stage[t], sx, sy, sz, entry, tj)) continue;
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

__global__ void __launch_bounds__(NB_WARPS * 32) k_neighbors(Bufs b, const int *gate)
{
    GATE;
    __shared__ float4 stage[NB_WARPS][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * NB_WARPS + w;
    if (c >= b.ncell_total) return;   // the whole warp
    const int s0 = b.cstart[c], s1 = b.cstart[c + 1];
    if (s0 == s1) return;
    nb_scan_cell(b, c, s0, s1, stage[w], lane);
}

// Half-size cells hold about 11 particles, too few for one lane per particle.
// This form gives the lanes candidates instead.
//
// A warp takes one cell. It flattens the candidates of the cell's
// neighbour cells (ascending key, then slot), and takes the cell's particles
// in groups of NG_G. For each group:
// * Every batch of 32 candidates is tested against the group's bounding box,
//   widened to the list radius. About half of the 125-cell stencil survives
//   for a half cell, against 27 cells' worth of candidates for a full cell.
// * The survivors are compacted in order into a staging area.
// * Each full stage of 32 runs one round per particle of the group: every
//   lane tests its candidate against that particle. Ballots place the hits in
//   scan order.
// * The group's lists are collected in shared memory as 16-bit entries (the
//   neighbour cell in the table, the offset in the cell, the contact-only
//   flag), owned entries from the front and the others from the back.
// * The lists are then written out row by row, the group's particles side by
//   side (32 / 8 = 4 rows per store for a full group), instead of one
//   scattered column entry per lane.
// A cell with a neighbour cell of more than 256 particles (beyond the 8-bit
// offset) is scanned by the lane-per-particle routine instead.  Either way
// the lists come out exactly as the lane-per-particle kernel writes them from
// the same cells: the same entries in the same order, the same counts and
// flags.
constexpr int NG_G = 8;        // particles per group
constexpr int NG_TAB = 128;    // neighbour-cell table entries (>= ADJ)
constexpr int NG_STAGE = 64;   // staged candidates (one batch on top of a partial stage)
constexpr int NG_MAX_WARPS = 4;
constexpr int NG_OFF = 256;    // largest neighbour cell of the 16-bit entries

struct NgShared {
    float4 sa[NG_STAGE];       // staged candidates: record,
    int sj[NG_STAGE];          //   slot,
    float sr[NG_STAGE];        //   radius where it can be a contact partner, else 0
    int sq[NG_STAGE];          //   neighbour cell << 8 | offset in it
    int pre[NG_TAB + 1];       // candidates before each neighbour cell (flattened index)
    int js[NG_TAB];            // first slot of each neighbour cell
    uint8_t code[NG_TAB];      // its offset code (ox+2) + 5 (oy+2) + 25 (oz+2) < 125
    float4 ai[NG_G];           // the group's records,
    float ri[NG_G];            //   rigid radii
};

// list-buffer row stride (16-bit entries): stride % 64 == 8 puts the rows
// of consecutive particles 16 bytes (4 banks) apart
__host__ __device__ constexpr int ng_stride(int cap) { return cap + ((72 - cap % 64) % 64); }
__host__ __device__ constexpr size_t ng_head() { return (sizeof(NgShared) + 15) / 16 * 16; }
__host__ __device__ constexpr size_t ng_warp_bytes(int cap)
{
    return ng_head() + (size_t)NG_G * ng_stride(cap) * sizeof(uint16_t);
}

__global__ void __launch_bounds__(NG_MAX_WARPS * 32) k_neighbors_grp(Bufs b, const int *gate)
{
    GATE;
    extern __shared__ __align__(16) unsigned char ng_smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int c = blockIdx.x * nw + w;
    if (c >= b.ncell_total) return;   // the whole warp
    const int s0 = b.cstart[c], s1 = b.cstart[c + 1];
    if (s0 == s1) return;
    const int cap = b.cap, stride = ng_stride(cap);
    unsigned char *mine = ng_smem + (size_t)w * ng_warp_bytes(cap);
    NgShared &S = *reinterpret_cast<NgShared *>(mine);
    uint16_t *buf = reinterpret_cast<uint16_t *>(mine + ng_head());
    const unsigned FULL = 0xffffffffu, lt = (1u << lane) - 1u;

    // neighbour-cell table (valid codes are a prefix of the row)
    const int *adj = b.cell_adj + (long long)c * ADJ;
    int total = 0, nq = 0;
    bool fat = false;
    for (int q0 = 0; q0 < ADJ; q0 += 32) {
        const int q = q0 + lane;
        const int code = q < ADJ ? adj[q] : -1;
        int cnt = 0, js = 0;
        if (code >= 0) {
            const int key = code >> 7;
            js = b.cstart[key];
            cnt = b.cstart[key + 1] - js;
        }
        fat = fat || __any_sync(FULL, cnt > NG_OFF);
        int v = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, v, o);
            if (lane >= o) v += t;
        }
        if (code >= 0) {
            S.pre[q] = total + v - cnt;
            S.js[q] = js;
            S.code[q] = (uint8_t)(code & 127);
        }
        total += __shfl_sync(FULL, v, 31);
        const unsigned vm = __ballot_sync(FULL, code >= 0);
        nq += __popc(vm);
        if (vm != FULL) break;
    }
    if (fat) {
        // the list buffer serves as the routine's stage (512 bytes)
        nb_scan_cell(b, c, s0, s1, reinterpret_cast<float4 *>(buf), lane);
        return;
    }
    if (lane == 0) S.pre[nq] = total;
    __syncwarp();

    const Inst &I = b.inst[b.pinst[b.perm[s0]]];   // a cell belongs to one instance
    const int base = b.cstart[I.cell_base];           // first slot of the instance
    const long long Np = b.Npad;
    const float rb2_box = I.rb2f * 1.001f;   // conservative: the pair test decides
    const float two_hs = (float)(2.0 * I.half_skin);
    const float cx = I.csf[0], cy = I.csf[1], cz = I.csf[2];
    const float BIG = 3.0e38f;

    for (int g0 = s0; g0 < s1; g0 += NG_G) {
        const int P = min(NG_G, s1 - g0);
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        int t = T_FLUID;
        float r = 0.f;
        if (lane < P) {
            a = b.A32[g0 + lane];
            t = b.stype[g0 + lane];
            r = (t == T_RIGID) ? (float)b.R[b.perm[g0 + lane]] : 0.f;
            S.ai[lane] = a;
            S.ri[lane] = r;
        }
        float lx = lane < P ? a.x : BIG, ly = lane < P ? a.y : BIG, lz = lane < P ? a.z : BIG;
        float hx = lane < P ? a.x : -BIG, hy = lane < P ? a.y : -BIG, hz = lane < P ? a.z : -BIG;
        float rg = r;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {   // lanes >= NG_G hold the neutral values
            lx = fminf(lx, __shfl_xor_sync(FULL, lx, o));
            ly = fminf(ly, __shfl_xor_sync(FULL, ly, o));
            lz = fminf(lz, __shfl_xor_sync(FULL, lz, o));
            hx = fmaxf(hx, __shfl_xor_sync(FULL, hx, o));
            hy = fmaxf(hy, __shfl_xor_sync(FULL, hy, o));
            hz = fmaxf(hz, __shfl_xor_sync(FULL, hz, o));
            rg = fmaxf(rg, __shfl_xor_sync(FULL, rg, o));
        }
        lx = __shfl_sync(FULL, lx, 0); ly = __shfl_sync(FULL, ly, 0); lz = __shfl_sync(FULL, lz, 0);
        hx = __shfl_sync(FULL, hx, 0); hy = __shfl_sync(FULL, hy, 0); hz = __shfl_sync(FULL, hz, 0);
        rg = __shfl_sync(FULL, rg, 0);
        const bool grp_rigid = __any_sync(FULL, lane < P && t == T_RIGID);
        __syncwarp();

        int nf[NG_G], m[NG_G];
        bool rig[NG_G];
#pragma unroll
        for (int p = 0; p < NG_G; ++p) { nf[p] = 0; m[p] = 0; rig[p] = false; }

        // one round per particle over the first nv staged candidates
        auto rounds = [&](int nv) {
            float4 Aj = make_float4(0.f, 0.f, 0.f, 0.f);
            int j = -1, tj = T_FLUID;
            uint32_t e16 = 0;
            float rj = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
            if (lane < nv) {
                Aj = S.sa[lane];
                j = S.sj[lane];
                rj = S.sr[lane];
                e16 = (uint32_t)S.sq[lane];
                const int oc = S.code[e16 >> 8];
                tj = unpack_type(__float_as_uint(Aj.w));
                sx = (float)(oc % 5 - 2) * cx;
                sy = (float)((oc / 5) % 5 - 2) * cy;
                sz = (float)(oc / 25 - 2) * cz;
            }
#pragma unroll
            for (int p = 0; p < NG_G; ++p) {
                if (p < P) {
                    const float4 Ai = S.ai[p];
                    const int ti = unpack_type(__float_as_uint(Ai.w));
                    const int s = g0 + p;
                    bool hit = false;
                    uint32_t entry = e16;
                    if (lane < nv && j != s) {
                        const float dx = (Ai.x - Aj.x) - sx, dy = (Ai.y - Aj.y) - sy, dz = (Ai.z - Aj.z) - sz;
                        const float r2f = dx * dx + dy * dy + dz * dz;
                        if (r2f < I.rb2f) {
                            hit = true;
                        } else if (ti == T_RIGID && tj == T_RIGID) {
                            const float lim = (S.ri[p] + rj + two_hs) * 1.0001f;
                            entry |= 0x8000u;   // contact range only
                            hit = r2f < lim * lim;
                        }
                    }
                    const bool own = hit && pair_owned(s, j, base);
                    const unsigned mh = __ballot_sync(FULL, hit), mo = __ballot_sync(FULL, own);
                    const unsigned mr = __ballot_sync(FULL, hit && tj == T_RIGID);
                    // rank in scan order decides whether the entry fits, as
                    // the per-particle scan writes while nf + m < cap
                    if (hit && nf[p] + m[p] + __popc(mh & lt) < cap) {
                        const int pos = own ? nf[p] + __popc(mo & lt) : cap - 1 - (m[p] + __popc(mh & ~mo & lt));
                        buf[p * stride + pos] = (uint16_t)entry;
                    }
                    nf[p] += __popc(mo);
                    m[p] += __popc(mh & ~mo);
                    rig[p] = rig[p] || (mr != 0u);
                }
            }
            __syncwarp();
        };

        int nst = 0, qc = 0;
        for (int f0 = 0; f0 < total; f0 += 32) {
            const int f = f0 + lane;
            bool keep = false;
            float4 Aj = make_float4(0.f, 0.f, 0.f, 0.f);
            int j = 0, eq = 0, q = qc;
            float rj = 0.f;
            if (f < total) {
                while (S.pre[q + 1] <= f) ++q;
                const int off = f - S.pre[q];
                j = S.js[q] + off;
                eq = (q << 8) | off;
                const int oc = S.code[q];
                Aj = b.A32[j];
                const int tj = unpack_type(__float_as_uint(Aj.w));
                const float px = Aj.x + (float)(oc % 5 - 2) * cx, py = Aj.y + (float)((oc / 5) % 5 - 2) * cy,
                            pz = Aj.z + (float)(oc / 25 - 2) * cz;
                const float ex = fmaxf(fmaxf(lx - px, px - hx), 0.f), ey = fmaxf(fmaxf(ly - py, py - hy), 0.f),
                            ez = fmaxf(fmaxf(lz - pz, pz - hz), 0.f);
                const float d2 = ex * ex + ey * ey + ez * ez;
                float lim2 = rb2_box;
                if (grp_rigid && tj == T_RIGID) {
                    rj = (float)b.R[b.perm[j]];
                    const float L = (rg + rj + two_hs) * (1.0001f * 1.0005f);
                    lim2 = fmaxf(lim2, L * L);
                }
                keep = d2 < lim2;
            }
            qc = __shfl_sync(FULL, q, 31);   // the cell of this batch's last candidate
            const unsigned km = __ballot_sync(FULL, keep);
            if (keep) {
                const int pos = nst + __popc(km & lt);
                S.sa[pos] = Aj;
                S.sj[pos] = j;
                S.sq[pos] = eq;
                S.sr[pos] = rj;
            }
            nst += __popc(km);
            __syncwarp();
            if (nst >= 32) {
                rounds(32);
                // move the remainder to the front of the stage
                const bool mv = lane < nst - 32;
                float4 ma;
                int mj = 0, mq = 0;
                float mr = 0.f;
                if (mv) {
                    ma = S.sa[32 + lane];
                    mj = S.sj[32 + lane];
                    mq = S.sq[32 + lane];
                    mr = S.sr[32 + lane];
                }
                __syncwarp();
                if (mv) {
                    S.sa[lane] = ma;
                    S.sj[lane] = mj;
                    S.sq[lane] = mq;
                    S.sr[lane] = mr;
                }
                nst -= 32;
                __syncwarp();
            }
        }
        if (nst > 0) rounds(nst);

        // counts and flags of the group's particles
        int mynf = 0, mym = 0;
        bool myrig = false;
#pragma unroll
        for (int p = 0; p < NG_G; ++p)
            if (lane == p) { mynf = nf[p]; mym = m[p]; myrig = rig[p]; }
        int myn = 0;
        if (lane < P) {
            const int s = g0 + lane;
            myn = mynf + mym;
            if (mynf > b.capown || mym > b.capown) atomicOr(b.err, ERR_PAIR_CAP);
            if (myn > cap) atomicOr(b.err, ERR_NBR_CAP);
            b.nfirst[s] = min(mynf, min(cap, b.capown));
            b.ncnt[s] = min(myn, cap);
            b.nbflag[s] = myrig ? 1 : 0;
        }
        int maxn = lane < P ? min(myn, cap) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) maxn = max(maxn, __shfl_xor_sync(FULL, maxn, o));
        // write-out: lane = (row kr, particle p), the group's particles side
        // by side; without overflow the back region [cap - m, cap) moves
        // down to [nf, n) as it is
        const int L = P > 4 ? 8 : (P > 2 ? 4 : P);   // lanes per row (P = 1, 2, 4 or 8 after rounding up)
        const int lsh = L == 8 ? 3 : (L == 4 ? 2 : L - 1);
        const int p = lane & (L - 1), kr = lane >> lsh, R = 32 >> lsh;
        const int pnf = __shfl_sync(FULL, mynf, p), pm = __shfl_sync(FULL, mym, p);
        const int pn = pnf + pm, pcnt = min(pn, cap);
        const bool wp = p < P;
        for (int k0 = 0; k0 < maxn; k0 += R) {
            const int k = k0 + kr;
            if (wp && k < pcnt) {
                const int src = (pn > cap || k < pnf) ? k : cap - pm + (k - pnf);
                const uint32_t e = buf[p * stride + src];
                const int slot = S.js[(e >> 8) & 127u] + (int)(e & 255u);
                b.nbr[(long long)k * Np + g0 + p] = (int)((uint32_t)slot | ((e & 0x8000u) ? NB_FAR : 0u));
            }
        }
        __syncwarp();
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

// dynamic shared memory of the lane-per-candidate list kernel: at least one
// warp's buffers at the largest list capacity
constexpr size_t NG_SMEM_MAX = 200 * 1024;
static_assert(ng_warp_bytes(SDPD_MAX_NEIGHBORS) <= NG_SMEM_MAX, "list buffers of one warp exceed the limit");

void init_cell_kernels()
{
    cudaFuncSetAttribute(k_neighbors_grp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NG_SMEM_MAX);
}

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
        if (b.cell_sub == 2) {
            const size_t wb = ng_warp_bytes(b.cap);
            const int ngw = (int)std::min<size_t>(NG_MAX_WARPS, NG_SMEM_MAX / wb);
            k_neighbors_grp<<<nblk(nc, ngw), ngw * 32, ngw * wb, st>>>(b, gate);
        } else {
            k_neighbors<<<nblk(nc, NB_WARPS), NB_WARPS * 32, 0, st>>>(b, gate);
        }
        if (need_rev) k_rev<<<nblk(b.N, 128), 128, 0, st>>>(b, gate);
    }
    k_build_done<<<1, 1, 0, st>>>(b, gate);
}

}  // namespace sdpd
