// misa_kernels.cuh -- the CUDA kernels of the EAM lattice-list MD step.
//
// Hot path of MISA-MD (arXiv:2107.07866) re-designed for one GB300:
//   density pass   rho_i = sum_j f(r_ij)               (Sec. 2.2 step 1)
//   embedding      F'(rho_i)                           (Sec. 2.2 step 2)
//   force pass     F_i = sum_j [(F'_i + F'_j) f'(r) + phi'(r)] (x_j - x_i)/r
//                                                      (Eq. eam_force_ij, steps 3-5)
// over the lattice list (Sec. 3): array atoms are reached through the
// neighbour offset index (Alg. 1 part 1), run-away atoms through a short
// list that every nearby tile and every run-away scans (Alg. 1 parts 2-3,
// read symmetrically).  Every per-atom result is written by exactly one
// thread: a full-neighbour gather with no atomics on densities or forces.
//
// A CTA owns one tile of TX x TY x TZ cells at a time (persistent loop over
// tiles) and stages the displacements of the tile plus a 2-cell halo into
// shared memory as (ux, uy, uz, F') vectors, split by parity so that the 8
// lanes of a quarter warp read 128 contiguous bytes.  The FP32 path keeps the
// spline coefficients of the pass in shared memory for the whole launch.
#pragma once

#include <type_traits>

#include "misa_common.cuh"

namespace misa {

constexpr int kRaChunk = 128;  // run-away atoms staged per round in a tile CTA
// A walker that visits a run-away's or a site's run-away neighbours scans
// the whole list when the replica has at most this many run-aways (one
// load per entry), else its tile's index segment (two dependent loads per
// entry, but only the entries within reach).  Both visit the pairs inside
// rc in list order, so the results do not depend on the choice.
constexpr int kRaScanMax = 32;
constexpr int kRedFloats = 112; // block-reduction scratch: 33 floats, then 32 doubles from byte 192
constexpr double kRws = 1.1180339887498949;  // max distance to the nearest bcc site: sqrt(5)/2 (a0/2 units)

// ---------------------------------------------------------------------------
// arithmetic traits
// ---------------------------------------------------------------------------

template <typename T>
struct Arith;

template <>
struct Arith<float> {
    static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
    // split x into floor (as int) and fraction, with ALU adds only: round
    // (x - 0.5) to an integer by the 1.5*2^23 trick.  At an exact integer x
    // either neighbouring segment may be chosen (t = 0 or t = 1); the spline
    // is C1 there, so both give the same value.
    static __device__ __forceinline__ int split(float x, float &t)
    {
        const float magic = 12582912.0f;
        float y = __fadd_rn(__fsub_rn(x, 0.5f), magic);
        float fl = __fsub_rn(y, magic);
        t = __fsub_rn(x, fl);
        return __float_as_int(y) - 0x4B400000;
    }
};

// 1/sqrt(x) in FP64 for x in FP32's normal range (pair distances squared):
// an FP32 seed (conversions on the integer pipe) and two Newton steps
// y <- y - y (x y^2 - 1) / 2, each doubling the correct bits (24 -> 48 ->
// full precision, a few ulps of rounding).  FP64 runs at a small fraction
// of the FP32 rate on GB300; this takes 8 FP64 operations where an IEEE
// square root and division take several times that.
__device__ __forceinline__ double rsqrt_nr(double x)
{
    double y = f2d_bits(rsqrtf(d2f_bits(x)));
    double h = fma(x * y, y, -1.0);
    y = fma(-0.5 * y, h, y);
    h = fma(x * y, y, -1.0);
    return fma(-0.5 * y, h, y);
}

template <>
struct Arith<double> {
    static __device__ __forceinline__ double rsqrt(double x) { return rsqrt_nr(x); }
    static __device__ __forceinline__ int split(double x, double &t)
    {
        double fl = floor(x);
        t = x - fl;
        return (int)fl;
    }
};

// Compensated accumulator: Kahan summation in FP32, plain sum in FP64.
template <typename T>
struct Acc {
    T s = 0, c = 0;
    __device__ __forceinline__ void add(T v)
    {
        if constexpr (sizeof(T) == 4) {
            T y = v - c;
            T t = s + y;
            c = (t - s) - y;
            s = t;
        } else {
            s += v;
        }
    }
    __device__ __forceinline__ T value() const { return s - c; }
};

// ---------------------------------------------------------------------------
// spline tables (Sec. 4.1)
// ---------------------------------------------------------------------------
// Knot slopes of the local cubic Hermite reading (central differences, 4th
// order inside, 2nd order at the two outer knots of each end), then the
// power form of segment k in t = x/h - k:
//   S = ((a t + b) t + c) t + d,   S'(x) = (3a t^2 + 2b t + c) / h.

__device__ __forceinline__ double knot_slope(const double *y, int n, double h, int k)
{
    if (k == 0) return (-3.0 * y[0] + 4.0 * y[1] - y[2]) / (2.0 * h);
    if (k == n - 1) return (3.0 * y[n - 1] - 4.0 * y[n - 2] + y[n - 3]) / (2.0 * h);
    if (k == 1 || k == n - 2) return (y[k + 1] - y[k - 1]) / (2.0 * h);
    return (y[k - 2] - 8.0 * y[k - 1] + 8.0 * y[k + 1] - y[k + 2]) / (12.0 * h);
}

// tab_f, tab_phi, tab_F: value coefficients; tab_d0/tab_d1: derivative
// coefficients of f and phi with respect to r, (A, B, C) with S' = (A t + B) t + C.
template <typename T>
__global__ void k_spline_tables(const double *fk, const double *pk, const double *Fk, int n, double hr,
                                double hrho, Vec4<T> *tab_f, Vec4<T> *tab_phi, Vec4<T> *tab_F,
                                Vec4<T> *tab_d0, Vec2<T> *tab_d1)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == n - 1) {
        // one all-zero entry past the last segment: the FP32 gathers clamp
        // every index at or beyond rc to it
        tab_f[k] = tab_phi[k] = tab_F[k] = tab_d0[k] = Vec4<T>{0, 0, 0, 0};
        tab_d1[k] = Vec2<T>{0, 0};
    }
    if (k >= n - 1) return;
    double cf[4], cp[4], cF[4];
    const double *ys[3] = {fk, pk, Fk};
    double hs[3] = {hr, hr, hrho};
    double *cs[3] = {cf, cp, cF};
    for (int q = 0; q < 3; ++q) {
        const double *y = ys[q];
        double h = hs[q];
        double m0 = knot_slope(y, n, h, k) * h, m1 = knot_slope(y, n, h, k + 1) * h;
        double y0 = y[k], y1 = y[k + 1];
        cs[q][0] = 2.0 * (y0 - y1) + m0 + m1;
        cs[q][1] = 3.0 * (y1 - y0) - 2.0 * m0 - m1;
        cs[q][2] = m0;
        cs[q][3] = y0;
    }
    tab_f[k] = Vec4<T>{(T)cf[0], (T)cf[1], (T)cf[2], (T)cf[3]};
    tab_phi[k] = Vec4<T>{(T)cp[0], (T)cp[1], (T)cp[2], (T)cp[3]};
    tab_F[k] = Vec4<T>{(T)cF[0], (T)cF[1], (T)cF[2], (T)cF[3]};
    tab_d0[k] = Vec4<T>{(T)(3.0 * cf[0] / hr), (T)(2.0 * cf[1] / hr), (T)(cf[2] / hr), (T)(3.0 * cp[0] / hr)};
    tab_d1[k] = Vec2<T>{(T)(2.0 * cp[1] / hr), (T)(cp[2] / hr)};
}

// Embedding F(rho) and F'(rho); linear continuation above rho_max.
template <typename T>
__device__ __forceinline__ T embed(const Vec4<T> *__restrict__ tab, int nseg, T Srho, T rho_max, T rho, T &dF,
                                   unsigned &st)
{
    if (rho > rho_max) {
        Vec4<T> c = tab[nseg - 1];
        T S1 = c.x + c.y + c.z + c.w;
        T D1 = (3 * c.x + 2 * c.y + c.z) * Srho;
        dF = D1;
        st |= kStRhoExtrap;
        return S1 + D1 * (rho - rho_max);
    }
    if (!(rho > 0)) rho = 0;
    T t;
    int k = Arith<T>::split(rho * Srho, t);
    k = min(max(k, 0), nseg - 1);
    if (k == nseg - 1 && t > 1) t = 1;
    Vec4<T> c = tab[k];
    dF = ((3 * c.x * t + 2 * c.y) * t + c.z) * Srho;
    return ((c.x * t + c.y) * t + c.z) * t + c.w;
}

// ---------------------------------------------------------------------------
// gather arguments
// ---------------------------------------------------------------------------

// Per-shell constants of the offset index (shells of equal |n|, sorted).
struct ShellInfo {
    int nshell;              // shells within rc + 2 skin
    float thr[kMaxShell];    // rc^2 - n^2 (lattice units)
    float nrm[kMaxShell];    // |n|
    float xfrac[kMaxShell];  // |n| S = xint + xfrac, xfrac in [0, 1)
    int xoff[kMaxShell];     // xint - 0x4B400000 (bit offset of the rounding trick)
    double thr_d[kMaxShell];
};

template <typename T>
struct GatherArgs {
    const RepDesc *reps;    // replica table
    const int *tile_rep;    // replica of every global tile
    int ntiles;             // tiles of all replicas
    int nrep;
    const T *ux, *uy, *uz;  // displacement per site (pooled), lattice units; vacant = kVacant
    const T *fp;            // force pass input: F' per site
    T *fp_out;              // density pass output
    T *rho_out;             // density (energy mode) or null
    double *e_out;          // per-site energy (energy mode) or null
    T *ax, *ay, *az;        // acceleration out (A/fs^2)
    double *vx, *vy, *vz;   // velocity (kick)
    const Vec4<T> *tab_f, *tab_phi, *tab_F, *tab_d0;
    const Vec2<T> *tab_d1;
    int nseg;
    int seg_lo;  // first segment an array-array pair can reach (r >= d_nn - 2 skin)
    T S;         // knot index per lattice unit of r: (a0/2)/h_r
    T Srho;      // 1/h_rho
    T rho_max;
    T rc2;       // rc^2, lattice units
    T rc_lat;
    T rfloor2;   // r_floor^2, lattice units
    // run-away lists (pooled; replica r owns [ra_base, ra_base + cap))
    const int *ra_home;     // home site, local to the replica
    const T *ra_ux, *ra_uy, *ra_uz;
    const T *ra_fp;
    const int *tile_flag;   // per global tile
    DevScalars *sc;         // per replica
    double acc_conv;        // (eV/A) -> (A/fs^2): 9.6485e-3 / m
    int kick;
    // FP32 gathers: per site, which candidates of the sparse shells (|n|^2 > 12)
    // the density pass found inside rc (bit k - first sparse candidate); the
    // force pass evaluates only those.  mask_ok = 0: evaluate all of them.
    unsigned long long *bmask;
    int mask_ok;
    // per-tile run-away index of this pass's tile map: tile t stages the
    // sorted list indices [ra_toff[t], ra_toff[t] + ra_tcnt[t]) of ra_tlist
    // when tile_flag[t] == 1 (2: the index overflowed, scan the whole list)
    const int *ra_toff, *ra_tcnt, *ra_tlist;
    unsigned long long tex_f, tex_d0, tex_d1;  // texture objects over tab_f, tab_d0, tab_d1
    // alloys (several species; null / zero for one): species per atom id,
    // run-away atom ids, and the per-species tables (nknot entries each, the
    // last all zero) through texture objects: density value and derivative
    // per species, pair derivative per unordered species pair; embedding and
    // pair values (energy evaluations) from global memory
    const int8_t *atype;
    const int *sid, *ra_id;  // atom id per site (-1: vacant), per run-away
    int nsp, nknot;
    int amaj;  // the dominant species: the density pass keeps its density window in shared memory
    unsigned long long tex_afv, tex_afd, tex_apd;
    const Vec4<T> *al_tFv, *al_tpv;
    const Vec4<T> *al_tfv;  // density values per species (the table of tex_afv)
    // neighbour offset index for this tile shape: per parity, per lattice
    // vector: (shared-memory slot displacement as int bits, 2 n_x, 2 n_y, 2 n_z)
    float4 off[2][kNVec];
    // the same for the FP32 two-site gathers, components paired:
    // (2nx, 2nx, 2ny, 2ny), (2nz, 2nz, slot displacement bits, 0)
    float4 offp[2][kNVec][2];
    ShellInfo sh;
};

template <int TX, int TY, int TZ>
struct Tile {
    static constexpr int SX = TX + 4, SY = TY + 4, SZ = TZ + 4;
    static constexpr int PLANE = SX * SY * SZ;
    static constexpr int PER_PAR = TX * TY * TZ;
    static constexpr int NT = 2 * PER_PAR;  // one thread per site
};

template <typename T>
__host__ __device__ inline size_t tile_smem_bytes(int tx, int ty, int tz)
{
    return sizeof(Vec4<T>) * 2 * (size_t)(tx + 4) * (ty + 4) * (tz + 4);
}

struct RaStage {
    int cnt, next;
};

__device__ __forceinline__ int wrap_cell(int g, int n)
{
    if (g < 0) g += n;
    while (g >= n) g -= n;
    return g;
}

// Global tile -> replica, its descriptor and the tile's cell origin.
struct TileLoc {
    int rep;
    RepDesc rd;
    int c0x, c0y, c0z;
};

__device__ __forceinline__ TileLoc finish_locate(TileLoc L, int tile, int TX, int TY, int TZ)
{
    const int lt = tile - L.rd.tile_base;
    const int tix = lt % L.rd.ntx, tiy = (lt / L.rd.ntx) % L.rd.nty, tiz = lt / (L.rd.ntx * L.rd.nty);
    L.c0x = tix * TX;
    L.c0y = tiy * TY;
    L.c0z = tiz * TZ;
    return L;
}

__device__ __forceinline__ TileLoc locate_tile(const RepDesc *reps, const int *tile_rep, int tile, int TX, int TY,
                                               int TZ)
{
    TileLoc L;
    L.rep = tile_rep[tile];
    L.rd = reps[L.rep];
    return finish_locate(L, tile, TX, TY, TZ);
}

// ---------------------------------------------------------------------------
// tile staging
// ---------------------------------------------------------------------------

// Loads (ux, uy, uz, F') of the tile at (c0x, c0y, c0z) of replica rd plus a
// 2-cell periodic halo into sU, split by parity.  Returns max |u| over the
// occupied staged sites (lattice units), block-wide.
template <typename T, int TX, int TY, int TZ, bool WITH_FP>
__device__ __forceinline__ T stage_tile(const GatherArgs<T> &a, const TileLoc &L, Vec4<T> *sU, float *sred)
{
    using G = Tile<TX, TY, TZ>;
    T umax2 = 0;
    for (int q = threadIdx.x; q < 2 * G::PLANE; q += G::NT) {
        const int p = q & 1;
        const int r = q >> 1;
        const int x = r % G::SX;
        const int yz = r / G::SX;
        const int y = yz % G::SY;
        const int z = yz / G::SY;
        const int gx = wrap_cell(L.c0x - 2 + x, L.rd.nx);
        const int gy = wrap_cell(L.c0y - 2 + y, L.rd.ny);
        const int gz = wrap_cell(L.c0z - 2 + z, L.rd.nz);
        const long long sid = L.rd.site_base + (((long long)gz * L.rd.ny + gy) * L.rd.nx + gx) * 2 + p;
        Vec4<T> v;
        v.x = a.ux[sid];
        v.y = a.uy[sid];
        v.z = a.uz[sid];
        v.w = WITH_FP ? a.fp[sid] : (T)0;
        const T u2 = v.x * v.x + v.y * v.y + v.z * v.z;
        if (v.x < (T)(0.5f * kVacant)) umax2 = umax2 > u2 ? umax2 : u2;
        sU[p * G::PLANE + (z * G::SY + y) * G::SX + x] = v;
    }
    float m = (float)umax2;
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        float w = threadIdx.x < (G::NT >> 5) ? sred[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) w = fmaxf(w, __shfl_xor_sync(0xffffffffu, w, o));
        if (threadIdx.x == 0) sred[32] = w;
    }
    __syncthreads();
    // round up by one FP32 ulp so that rounding never prunes a needed shell
    return (T)(sqrtf(sred[32]) * 1.000001f);
}

// Home lattice coordinates of run-away j of replica rd (home site h)
// relative to the tile origin (c0x, c0y, c0z) of a tx x ty x tz tile -- the
// nearest periodic image to the tile centre -- and whether its home cell
// lies within 3 cells of the tile (reach rc + skin + the Wigner-Seitz
// radius): the run-aways a tile stages.
__device__ __forceinline__ bool ra_in_tile_rt(const RepDesc &rd, int h, int c0x, int c0y, int c0z, int tx, int ty,
                                              int tz, int &hx, int &hy, int &hz)
{
    const int x2 = h % (2 * rd.nx);
    const int rest = h / (2 * rd.nx);
    const int cy = rest % rd.ny, cz = rest / rd.ny;
    const int par = x2 & 1, cx = x2 >> 1;
    int dx = cx - c0x - tx / 2, dy = cy - c0y - ty / 2, dz = cz - c0z - tz / 2;
    dx -= rd.nx * (int)floorf((dx + 0.5f * rd.nx) / rd.nx);
    dy -= rd.ny * (int)floorf((dy + 0.5f * rd.ny) / rd.ny);
    dz -= rd.nz * (int)floorf((dz + 0.5f * rd.nz) / rd.nz);
    dx += tx / 2; dy += ty / 2; dz += tz / 2;
    hx = 2 * dx + par;
    hy = 2 * dy + par;
    hz = 2 * dz + par;
    return dx >= -3 && dx < tx + 3 && dy >= -3 && dy < ty + 3 && dz >= -3 && dz < tz + 3;
}

template <int TX, int TY, int TZ>
__device__ __forceinline__ bool ra_in_tile(const RepDesc &rd, int h, int c0x, int c0y, int c0z, int &hx, int &hy,
                                           int &hz)
{
    return ra_in_tile_rt(rd, h, c0x, c0y, c0z, TX, TY, TZ, hx, hy, hz);
}

// Stages the next chunk of the replica's run-away atoms whose home cell lies
// within 3 cells of the tile, in list order, as (home lattice coords
// relative to the tile origin, u, F').  A tile with an index entry
// (tile_flag 1) copies its sorted entries; otherwise warp 0 scans the whole
// list.  Returns the staged count (block-uniform); pos advances, reaching
// nra when nothing is left.
template <typename T, int TX, int TY, int TZ, bool WITH_FP>
__device__ __forceinline__ int stage_runaways(const GatherArgs<T> &a, const TileLoc &L, int tile, int nra, int &pos,
                                              int4 *sRh, Vec4<T> *sRu, RaStage *st)
{
    const RepDesc &rd = L.rd;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int cnt = 0;
        int p0 = pos;
        if (a.tile_flag[tile] == 1) {
            // the tile's index entries: list indices in ascending order
            const int n = a.ra_tcnt[tile], off = a.ra_toff[tile];
            cnt = min(n - p0, kRaChunk);
            for (int q = lane; q < cnt; q += 32) {
                const int j = a.ra_tlist[off + p0 + q];
                int hx, hy, hz;
                ra_in_tile<TX, TY, TZ>(rd, a.ra_home[rd.ra_base + j], L.c0x, L.c0y, L.c0z, hx, hy, hz);
                sRh[q] = make_int4(hx, hy, hz, a.atype ? (int)a.atype[a.ra_id[rd.ra_base + j]] : 0);
                Vec4<T> u;
                u.x = a.ra_ux[rd.ra_base + j];
                u.y = a.ra_uy[rd.ra_base + j];
                u.z = a.ra_uz[rd.ra_base + j];
                u.w = WITH_FP ? a.ra_fp[rd.ra_base + j] : (T)0;
                sRu[q] = u;
            }
            p0 = p0 + cnt >= n ? nra : p0 + cnt;
        } else {
            while (p0 < nra && cnt < kRaChunk) {
                const int j = p0 + lane;
                bool take = false;
                int hx = 0, hy = 0, hz = 0;
                if (j < nra) take = ra_in_tile<TX, TY, TZ>(rd, a.ra_home[rd.ra_base + j], L.c0x, L.c0y, L.c0z, hx, hy, hz);
                const unsigned bal = __ballot_sync(0xffffffffu, take);
                const int room = kRaChunk - cnt;
                const int rank = __popc(bal & ((1u << lane) - 1u));
                if (take && rank < room) {
                    // w: the run-away's species (alloys)
                    sRh[cnt + rank] = make_int4(hx, hy, hz, a.atype ? (int)a.atype[a.ra_id[rd.ra_base + j]] : 0);
                    Vec4<T> u;
                    u.x = a.ra_ux[rd.ra_base + j];
                    u.y = a.ra_uy[rd.ra_base + j];
                    u.z = a.ra_uz[rd.ra_base + j];
                    u.w = WITH_FP ? a.ra_fp[rd.ra_base + j] : (T)0;
                    sRu[cnt + rank] = u;
                }
                const int ntake = __popc(bal);
                if (ntake <= room) {
                    cnt += ntake;
                    p0 += 32;
                } else {
                    // chunk full: resume at the first lane that did not fit
                    unsigned b = bal;
                    for (int q = 0; q < room; ++q) b &= b - 1;
                    p0 += __ffs(b) - 1;
                    cnt += room;
                }
            }
            if (p0 > nra) p0 = nra;
        }
        if (lane == 0) {
            st->cnt = cnt;
            st->next = p0;
        }
    }
    __syncthreads();
    const int c = st->cnt;
    pos = st->next;
    return c;
}

// ---------------------------------------------------------------------------
// pair geometry
// ---------------------------------------------------------------------------
// Array pair through offset vector n of shell s: q = (2n + d).d with
// d = u_j - u_i, so r^2 = n^2 + q.  Both atoms are within the skin of their
// sites, so r >= |n_1| - 2 skin > 1 A: no r floor is needed here.
// FP32: the spline argument is |n| S + (r - |n|) S with r - |n| = q/(r + |n|)
// (small, full relative precision) and the per-shell split
// |n| S = xint + xfrac, so the segment and t keep full FP32 precision
// instead of the ~1e-4 absolute error of r S near 2000.

template <typename T>
struct ShellRegs {
    T n2, thr, nrm, xfrac;
    int xoff;
};

template <typename T>
__device__ __forceinline__ int shell_arg(const ShellRegs<T> &sh, T q, T S, int seglo, int nseg1, T &t, T &rinv)
{
    const T r2 = sh.n2 + q;
    if constexpr (sizeof(T) == 4) {
        const float rs = rsqrtf(r2);
        rinv = rs;
        const float r = r2 * rs;
        const float dr = __fdividef(q, r + sh.nrm);
        const float x = fmaf(dr, S, sh.xfrac);
        const float y = __fadd_rn(__fsub_rn(x, 0.5f), 12582912.0f);
        const float fl = __fsub_rn(y, 12582912.0f);
        t = __fsub_rn(x, fl);
        return min(max(__float_as_int(y) + sh.xoff, seglo), nseg1);
    } else {
        rinv = rsqrt_nr(r2);
        const double r = r2 * rinv;
        const double x = r * S;
        const double fl = floor(x);
        t = x - fl;
        return min(max((int)fl, seglo), nseg1);
    }
}

// per-shell constants into registers (shell index known at compile time)
template <typename T, int SH>
__device__ __forceinline__ ShellRegs<T> shell_regs(const ShellInfo &sh)
{
    ShellRegs<T> r;
    constexpr int N2 = kLVec.shell_n2[SH];
    r.n2 = (T)N2;
    r.thr = sizeof(T) == 4 ? (T)sh.thr[SH] : (T)sh.thr_d[SH];
    r.nrm = (T)sh.nrm[SH];
    r.xfrac = (T)sh.xfrac[SH];
    r.xoff = sh.xoff[SH];
    return r;
}

// Spline argument from r^2 directly (run-away pairs: the offset is not a
// shell constant); clamps r at r_floor.
template <typename T>
__device__ __forceinline__ void direct_arg(T r2, T S, T rfloor2, int &seg, T &t, T &rinv, bool &floor_hit)
{
    floor_hit = r2 < rfloor2;
    r2 = floor_hit ? rfloor2 : r2;
    T rs = Arith<T>::rsqrt(r2);
    rinv = rs;
    const T r = r2 * rs;
    seg = Arith<T>::split(r * S, t);
}

template <typename T>
__device__ __forceinline__ int clamp_seg(int seg, int nseg, T &t)
{
    if (seg < 0) {
        t = 0;
        return 0;
    }
    if (seg > nseg - 1) {
        t = 1;
        return nseg - 1;
    }
    return seg;
}

// shared-memory carve-up of the tile kernels
// per-replica values a tile kernel reads at every tile, cached in shared
// memory for batches of up to kRepSmem replicas
constexpr int kRepSmem = 64;
struct RepCache {
    RepDesc rd;
    double dt;
    int n_ra;
    int pad;
};

template <typename T>
struct GatherSmem {
    RepCache *rep;
    float4 *off;
    Vec4<T> *u;
    int4 *rh;
    Vec4<T> *ru;
    float *red;
    RaStage *st;
};

template <typename T, int TX, int TY, int TZ>
__device__ __forceinline__ GatherSmem<T> carve(unsigned char *smem, size_t off, int nbuf)
{
    GatherSmem<T> g;
    off = (off + 255) & ~(size_t)255;
    g.rep = reinterpret_cast<RepCache *>(smem + off);
    off += sizeof(RepCache) * kRepSmem;
    g.off = reinterpret_cast<float4 *>(smem + off);
    off += sizeof(float4) * 2 * kNVec;
    g.u = reinterpret_cast<Vec4<T> *>(smem + off);
    off += sizeof(Vec4<T>) * 2 * Tile<TX, TY, TZ>::PLANE * nbuf;
    g.rh = reinterpret_cast<int4 *>(smem + off);
    off += sizeof(int4) * kRaChunk;
    g.ru = reinterpret_cast<Vec4<T> *>(smem + off);
    off += sizeof(Vec4<T>) * kRaChunk;
    g.red = reinterpret_cast<float *>(smem + off);
    off += sizeof(float) * kRedFloats;
    g.st = reinterpret_cast<RaStage *>(smem + off);
    return g;
}

// Copies the replica table and each replica's dt and run-away count into
// shared memory (batches of up to kRepSmem replicas; larger batches read
// them from global memory at every tile).
template <typename T>
__device__ __forceinline__ void fill_rep_cache(const GatherArgs<T> &a, RepCache *rc)
{
    if (a.nrep > kRepSmem) return;
    for (int r = threadIdx.x; r < a.nrep; r += blockDim.x) {
        RepCache c;
        c.rd = a.reps[r];
        c.dt = a.sc[r].dt;
        c.n_ra = a.sc[r].n_ra;
        c.pad = 0;
        rc[r] = c;
    }
}

template <typename T>
__device__ __forceinline__ TileLoc locate_cached(const GatherArgs<T> &a, const RepCache *rc, int tile, int TX, int TY,
                                                 int TZ, double &dt, int &nra)
{
    TileLoc L;
    L.rep = a.tile_rep[tile];
    if (a.nrep <= kRepSmem) {
        L.rd = rc[L.rep].rd;
        dt = rc[L.rep].dt;
        nra = rc[L.rep].n_ra;
    } else {
        L.rd = a.reps[L.rep];
        dt = a.sc[L.rep].dt;
        nra = a.sc[L.rep].n_ra;
    }
    return finish_locate(L, tile, TX, TY, TZ);
}

// FP32 density tiles are double-buffered (the next tile streams in by
// cp.async while the current one is computed).  The force pass and the FP64
// path stage synchronously: they are issue-bound, and the prefetch measured
// slower there.
template <typename T>
__host__ __device__ constexpr int tile_buffers()
{
    return sizeof(T) == 4 ? 2 : 1;
}
constexpr int kForceBuffers = 1;

template <typename T>
__host__ __device__ inline size_t gather_smem_bytes(size_t table_bytes, int tx, int ty, int tz, int nbuf)
{
    size_t off = (table_bytes + 255) & ~(size_t)255;
    off += sizeof(RepCache) * kRepSmem;
    off += sizeof(float4) * 2 * kNVec;
    off += tile_smem_bytes<T>(tx, ty, tz) * nbuf;
    off += sizeof(int4) * kRaChunk + sizeof(Vec4<T>) * kRaChunk + sizeof(float) * kRedFloats + sizeof(RaStage);
    return off;
}

// ---------------------------------------------------------------------------
// asynchronous tile staging (FP32 path): cp.async 4-byte copies of the
// displacement (and F') of every tile + halo slot straight into shared memory
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int TX, int TY, int TZ, bool WITH_FP>
__device__ __forceinline__ void issue_tile(const GatherArgs<float> &a, const RepCache *rc, Vec4<float> *sU, int tile)
{
    using G = Tile<TX, TY, TZ>;
    double dt_;
    int nra_;
    const TileLoc L = locate_cached(a, rc, tile, TX, TY, TZ, dt_, nra_);
    for (int q = threadIdx.x; q < 2 * G::PLANE; q += G::NT) {
        const int p = q & 1;
        const int r = q >> 1;
        const int x = r % G::SX;
        const int yz = r / G::SX;
        const int y = yz % G::SY;
        const int z = yz / G::SY;
        const int gx = wrap_cell(L.c0x - 2 + x, L.rd.nx);
        const int gy = wrap_cell(L.c0y - 2 + y, L.rd.ny);
        const int gz = wrap_cell(L.c0z - 2 + z, L.rd.nz);
        const long long sid = L.rd.site_base + (((long long)gz * L.rd.ny + gy) * L.rd.nx + gx) * 2 + p;
        Vec4<float> *d = sU + p * G::PLANE + (z * G::SY + y) * G::SX + x;
        cp_async4(&d->x, a.ux + sid);
        cp_async4(&d->y, a.uy + sid);
        cp_async4(&d->z, a.uz + sid);
        if (WITH_FP) cp_async4(&d->w, a.fp + sid);
    }
}

// max |u| over the occupied slots of a staged tile, block-wide
template <int TX, int TY, int TZ>
__device__ __forceinline__ float tile_umax(const Vec4<float> *sU, float *sred)
{
    using G = Tile<TX, TY, TZ>;
    float umax2 = 0.f;
    for (int q = threadIdx.x; q < 2 * G::PLANE; q += G::NT) {
        const Vec4<float> v = sU[q];
        const float u2 = v.x * v.x + v.y * v.y + v.z * v.z;
        if (v.x < 0.5f * kVacant) umax2 = fmaxf(umax2, u2);
    }
    for (int o = 16; o > 0; o >>= 1) umax2 = fmaxf(umax2, __shfl_xor_sync(0xffffffffu, umax2, o));
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = umax2;
    __syncthreads();
    if (threadIdx.x < 32) {
        float w = threadIdx.x < (G::NT >> 5) ? sred[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) w = fmaxf(w, __shfl_xor_sync(0xffffffffu, w, o));
        if (threadIdx.x == 0) sred[32] = w;
    }
    __syncthreads();
    return sqrtf(sred[32]) * 1.000001f;
}

// ---------------------------------------------------------------------------
// shell loops over the offset index
// ---------------------------------------------------------------------------
// Shells are visited in order of |n| and stop at the first one beyond
// lim = rc + |u_i| + max_tile |u_j|.  Shells up to n^2 = 12 (the 58
// neighbours of the crystal) are evaluated without a branch: a candidate
// outside rc is computed and masked (its segment index is clamped, so the
// arithmetic stays finite); farther shells branch, as almost all of their
// candidates fall outside rc.

template <typename T, int SH>
__device__ __forceinline__ void density_shells(const ShellInfo &shc, const float4 *__restrict__ po,
                                               const Vec4<T> *__restrict__ su, int slot, const Vec4<T> &ui, T lim2, T S,
                                               int seglo, int nseg1, const Vec4<T> *__restrict__ tabf, Acc<T> &rho)
{
    if constexpr (SH < kLVec.nshell) {
        constexpr int KB = kLVec.shell_begin[SH], KE = kLVec.shell_begin[SH + 1];
        constexpr int N2 = kLVec.shell_n2[SH];
        constexpr bool dense = N2 <= 12;
        if (SH >= shc.nshell || (T)N2 > lim2) return;
        const ShellRegs<T> sh = shell_regs<T, SH>(shc);
        T part = 0;
#pragma unroll 2
        for (int k = KB; k < KE; ++k) {
            const float4 o = po[k];
            const Vec4<T> uj = su[slot + __float_as_int(o.x)];
            const T dx = uj.x - ui.x, dy = uj.y - ui.y, dz = uj.z - ui.z;
            const T qq = (dx + (T)o.y) * dx + (dy + (T)o.z) * dy + (dz + (T)o.w) * dz;
            if (dense) {
                T t, rinv;
                const int seg = shell_arg<T>(sh, qq, S, seglo, nseg1, t, rinv);
                const Vec4<T> c = tabf[seg];
                const T v = ((c.x * t + c.y) * t + c.z) * t + c.w;
                part += qq < sh.thr ? v : (T)0;
            } else if (qq < sh.thr) {
                T t, rinv;
                const int seg = shell_arg<T>(sh, qq, S, seglo, nseg1, t, rinv);
                const Vec4<T> c = tabf[seg];
                part += ((c.x * t + c.y) * t + c.z) * t + c.w;
            }
        }
        rho.add(part);
        density_shells<T, SH + 1>(shc, po, su, slot, ui, lim2, S, seglo, nseg1, tabf, rho);
    }
}

template <typename T, int SH, bool ENERGY>
__device__ __forceinline__ void force_shells(const ShellInfo &shc, const float4 *__restrict__ po,
                                             const Vec4<T> *__restrict__ su, int slot, const Vec4<T> &ui, T lim2, T S,
                                             int seglo, int nseg1, const Vec4<T> *__restrict__ tab0, const Vec2<T> *__restrict__ tab1,
                                             const Vec4<T> *__restrict__ tabphi, Acc<T> &fx, Acc<T> &fy, Acc<T> &fz,
                                             double &ephi)
{
    if constexpr (SH < kLVec.nshell) {
        constexpr int KB = kLVec.shell_begin[SH], KE = kLVec.shell_begin[SH + 1];
        constexpr int N2 = kLVec.shell_n2[SH];
        constexpr bool dense = N2 <= 12;
        if (SH >= shc.nshell || (T)N2 > lim2) return;
        const ShellRegs<T> sh = shell_regs<T, SH>(shc);
        T px = 0, py = 0, pz = 0;
#pragma unroll 2
        for (int k = KB; k < KE; ++k) {
            const float4 o = po[k];
            const Vec4<T> uj = su[slot + __float_as_int(o.x)];
            const T dx = uj.x - ui.x, dy = uj.y - ui.y, dz = uj.z - ui.z;
            const T qq = (dx + (T)o.y) * dx + (dy + (T)o.z) * dy + (dz + (T)o.w) * dz;
            if (dense || qq < sh.thr) {
                T t, rinv;
                const int seg = shell_arg<T>(sh, qq, S, seglo, nseg1, t, rinv);
                const Vec4<T> c0 = tab0[seg];
                const Vec2<T> c1 = tab1[seg];
                const T dfr = (c0.x * t + c0.y) * t + c0.z;
                const T dph = (c0.w * t + c1.x) * t + c1.y;
                T sc_ = ((ui.w + uj.w) * dfr + dph) * rinv;
                if (dense) sc_ = qq < sh.thr ? sc_ : (T)0;
                px += sc_ * (dx + (T)0.5 * (T)o.y);
                py += sc_ * (dy + (T)0.5 * (T)o.z);
                pz += sc_ * (dz + (T)0.5 * (T)o.w);
                if (ENERGY) {
                    const Vec4<T> cp = tabphi[seg];
                    const double e = 0.5 * (double)(((cp.x * t + cp.y) * t + cp.z) * t + cp.w);
                    ephi += qq < sh.thr ? e : 0.0;
                }
            }
        }
        fx.add(px);
        fy.add(py);
        fz.add(pz);
        force_shells<T, SH + 1, ENERGY>(shc, po, su, slot, ui, lim2, S, seglo, nseg1, tab0, tab1, tabphi, fx, fy, fz, ephi);
    }
}

// ---------------------------------------------------------------------------
// run-away pairs inside a tile kernel (Alg. 1 parts 2-3, array side)
// ---------------------------------------------------------------------------
// Geometry from the home lattice vector (exact integers, minimum image) plus
// the two displacements; r is floored at r_floor.  Uses the full global
// tables (run-away pairs can come closer than any array pair).

template <typename T>
struct RaPair {
    bool in;
    int seg;
    T t, rinv, rx, ry, rz;
    bool floor_hit;
};

template <typename T>
__device__ __forceinline__ RaPair<T> ra_pair(const GatherArgs<T> &a, const RepDesc &rd, int4 h, const Vec4<T> &uj,
                                             const Vec4<T> &ui, int sx, int sy, int sz)
{
    RaPair<T> P;
    int nx_ = h.x - sx, ny_ = h.y - sy, nz_ = h.z - sz;
    // minimum image; a tile may be wider than the box, so the two sides can
    // be several box lengths apart
    const int Lx = 2 * rd.nx, Ly = 2 * rd.ny, Lz = 2 * rd.nz;
    while (nx_ > rd.nx) nx_ -= Lx;
    while (nx_ < -rd.nx) nx_ += Lx;
    while (ny_ > rd.ny) ny_ -= Ly;
    while (ny_ < -rd.ny) ny_ += Ly;
    while (nz_ > rd.nz) nz_ -= Lz;
    while (nz_ < -rd.nz) nz_ += Lz;
    // a run-away lies within the Wigner-Seitz radius sqrt(5)/2 of its home
    // and an array atom within the skin (< 0.64 lattice units) of its site,
    // so a pair inside rc has every component of n below rc + 1.76: the
    // integer test rejects the staged run-aways out of reach exactly
    const int K = (int)(a.rc_lat + (T)1.8);
    P.in = false;
    if (abs(nx_) > K || abs(ny_) > K || abs(nz_) > K) return P;
    const T dx = uj.x - ui.x, dy = uj.y - ui.y, dz = uj.z - ui.z;
    const T qq = (dx + (T)(2 * nx_)) * dx + (dy + (T)(2 * ny_)) * dy + (dz + (T)(2 * nz_)) * dz;
    const T r2 = (T)(nx_ * nx_ + ny_ * ny_ + nz_ * nz_) + qq;
    P.in = r2 < a.rc2;
    P.rx = dx + (T)nx_;
    P.ry = dy + (T)ny_;
    P.rz = dz + (T)nz_;
    if (P.in) {
        direct_arg<T>(r2, a.S, a.rfloor2, P.seg, P.t, P.rinv, P.floor_hit);
        P.seg = clamp_seg<T>(P.seg, a.nseg, P.t);
    }
    return P;
}

// ---------------------------------------------------------------------------
// density pass: rho_i, F'(rho_i)  (Sec. 2.2 steps 1-2)
// ---------------------------------------------------------------------------
// Each shell's terms are summed plainly (at most 24, similar magnitudes)
// and the shell sums are added with Kahan compensation.  One persistent CTA
// per SM walks the global tile list of all replicas.

template <typename T, int TX, int TY, int TZ, bool ENERGY>
__global__ void __launch_bounds__(2 * TX * TY * TZ, 1) k_density(const __grid_constant__ GatherArgs<T> a)
{
    using G = Tile<TX, TY, TZ>;
    constexpr bool DB = tile_buffers<T>() == 2;
    extern __shared__ __align__(32) unsigned char smem[];
    // FP32: the part of the f table that array pairs can reach, in shared memory
    const Vec4<T> *tabf = a.tab_f;
    size_t tbytes = 0;
    if constexpr (DB) {
        Vec4<T> *t = reinterpret_cast<Vec4<T> *>(smem);
        const int nwin = a.nseg - a.seg_lo;
        for (int k = threadIdx.x; k < nwin; k += G::NT) t[k] = a.tab_f[a.seg_lo + k];
        tabf = t - a.seg_lo;  // indexed by segment; segments >= seg_lo only
        tbytes = sizeof(Vec4<T>) * (size_t)nwin;
    }
    const GatherSmem<T> sm = carve<T, TX, TY, TZ>(smem, tbytes, tile_buffers<T>());
    for (int k = threadIdx.x; k < 2 * kNVec; k += G::NT) sm.off[k] = (&a.off[0][0])[k];
    fill_rep_cache<T>(a, sm.rep);
    __syncthreads();

    // this thread's site within a tile: parity-major, then (z, y, x)
    const int q = threadIdx.x;
    const int p = q / G::PER_PAR;
    const int rr = q % G::PER_PAR;
    const int lx = rr % TX, ly = (rr / TX) % TY, lz = rr / (TX * TY);
    const int slot = p * G::PLANE + ((lz + 2) * G::SY + (ly + 2)) * G::SX + (lx + 2);
    const float4 *po = sm.off + p * kNVec;
    const int nseg1 = a.nseg - 1;
    const int seglo = DB ? a.seg_lo : 0;
    unsigned st = 0;
    int buf = 0;
    if constexpr (DB) {
        if ((int)blockIdx.x < a.ntiles) issue_tile<TX, TY, TZ, false>(a, sm.rep, sm.u, blockIdx.x);
        cp_async_commit();
    }

    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        double dt_rep;
        int nra;
        const TileLoc L = locate_cached(a, sm.rep, tile, TX, TY, TZ, dt_rep, nra);
        Vec4<T> *cur = sm.u + buf * 2 * G::PLANE;
        T U;
        if constexpr (DB) {
            const int nxt = tile + gridDim.x;
            if (nxt < a.ntiles) issue_tile<TX, TY, TZ, false>(a, sm.rep, sm.u + (buf ^ 1) * 2 * G::PLANE, nxt);
            cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();
            U = tile_umax<TX, TY, TZ>(cur, sm.red);
        } else {
            __syncthreads();
            U = stage_tile<T, TX, TY, TZ, false>(a, L, cur, sm.red);
        }
        const bool has_ra = a.tile_flag[tile] != 0 && nra > 0;
        const bool inbox = (L.c0x + lx < L.rd.nx) && (L.c0y + ly < L.rd.ny) && (L.c0z + lz < L.rd.nz);
        const Vec4<T> ui = cur[slot];
        const bool live = inbox && ui.x < (T)(0.5f * kVacant);
        Acc<T> rho;
        if (live) {
            const T lim = a.rc_lat + sqrt(ui.x * ui.x + ui.y * ui.y + ui.z * ui.z) + U;
            density_shells<T, 0>(a.sh, po, cur, slot, ui, lim * lim, a.S, seglo, nseg1, tabf, rho);
        }
        if (has_ra) {
            int pos = 0;
            const int sx = 2 * lx + p, sy = 2 * ly + p, sz = 2 * lz + p;
            while (true) {
                __syncthreads();
                const int cnt = stage_runaways<T, TX, TY, TZ, false>(a, L, tile, nra, pos, sm.rh, sm.ru, sm.st);
                if (cnt == 0) break;
                if (live) {
                    for (int j = 0; j < cnt; ++j) {
                        const RaPair<T> P = ra_pair<T>(a, L.rd, sm.rh[j], sm.ru[j], ui, sx, sy, sz);
                        if (P.in) {
                            if (P.floor_hit) st |= kStRfloor;
                            const Vec4<T> c = a.tab_f[P.seg];
                            rho.add(((c.x * P.t + c.y) * P.t + c.z) * P.t + c.w);
                        }
                    }
                }
                if (pos >= nra) break;
            }
        }
        if (live) {
            const long long sid =
                L.rd.site_base + (((long long)(L.c0z + lz) * L.rd.ny + (L.c0y + ly)) * L.rd.nx + (L.c0x + lx)) * 2 + p;
            const T rh = rho.value();
            T dF;
            const T Fv = embed<T>(a.tab_F, a.nseg, a.Srho, a.rho_max, rh, dF, st);
            a.fp_out[sid] = dF;
            if (ENERGY) {
                a.rho_out[sid] = rh;
                a.e_out[sid] = (double)Fv;
            }
        }
        if constexpr (DB) {
            buf ^= 1;
            __syncthreads();  // every read of cur is done before it is refilled
        }
    }
    if constexpr (DB) cp_async_wait<0>();
    if (st) atomicOr(&a.sc[0].status, st);
}

// Block max of |v|^2 -> one atomicMax of |v| on the replica's accumulator
// (non-negative doubles order like their bit patterns).  Block-uniform call.
template <int NT>
__device__ __forceinline__ void flush_vmax(double vmax2, float *sred, DevScalars *sc)
{
    double m = vmax2;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    double *smd = reinterpret_cast<double *>(sred) + 24;  // clear of the floats stage_tile uses
    __syncthreads();
    if ((threadIdx.x & 31) == 0) smd[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double w = 0.0;
        for (int k = 0; k < NT / 32; ++k) w = fmax(w, smd[k]);
        if (w > 0.0) atomicMax(&sc->vacc_bits, (unsigned long long)__double_as_longlong(sqrt(w)));
    }
}

// ---------------------------------------------------------------------------
// force pass (Eq. eam_force_ij) + closing half kick of velocity Verlet
// ---------------------------------------------------------------------------

template <typename T, int TX, int TY, int TZ, bool ENERGY>
__global__ void __launch_bounds__(2 * TX * TY * TZ, 1) k_force(const __grid_constant__ GatherArgs<T> a)
{
    using G = Tile<TX, TY, TZ>;
    constexpr bool DB = kForceBuffers == 2 && tile_buffers<T>() == 2;
    constexpr bool TSM = sizeof(T) == 4;  // tables in shared memory
    extern __shared__ __align__(32) unsigned char smem[];
    // FP32: the part of the f', phi' tables that array pairs can reach
    const Vec4<T> *tab0 = a.tab_d0;
    const Vec2<T> *tab1 = a.tab_d1;
    size_t tbytes = 0;
    if constexpr (TSM) {
        const int nwin = a.nseg - a.seg_lo;
        Vec4<T> *t0 = reinterpret_cast<Vec4<T> *>(smem);
        Vec2<T> *t1 = reinterpret_cast<Vec2<T> *>(smem + sizeof(Vec4<T>) * (size_t)nwin);
        for (int k = threadIdx.x; k < nwin; k += G::NT) {
            t0[k] = a.tab_d0[a.seg_lo + k];
            t1[k] = a.tab_d1[a.seg_lo + k];
        }
        tab0 = t0 - a.seg_lo;
        tab1 = t1 - a.seg_lo;
        tbytes = (sizeof(Vec4<T>) + sizeof(Vec2<T>)) * (size_t)nwin;
    }
    const GatherSmem<T> sm = carve<T, TX, TY, TZ>(smem, tbytes, DB ? 2 : 1);
    for (int k = threadIdx.x; k < 2 * kNVec; k += G::NT) sm.off[k] = (&a.off[0][0])[k];
    fill_rep_cache<T>(a, sm.rep);
    __syncthreads();

    const int q = threadIdx.x;
    const int p = q / G::PER_PAR;
    const int rr = q % G::PER_PAR;
    const int lx = rr % TX, ly = (rr / TX) % TY, lz = rr / (TX * TY);
    const int slot = p * G::PLANE + ((lz + 2) * G::SY + (ly + 2)) * G::SX + (lx + 2);
    const float4 *po = sm.off + p * kNVec;
    const int nseg1 = a.nseg - 1;
    const int seglo = TSM ? a.seg_lo : 0;
    unsigned st = 0;
    const T conv = (T)a.acc_conv;
    int buf = 0;
    if constexpr (DB) {
        if ((int)blockIdx.x < a.ntiles) issue_tile<TX, TY, TZ, true>(a, sm.rep, sm.u, blockIdx.x);
        cp_async_commit();
    }

    int cur_rep = -1;
    double vmax2 = 0.0;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        double dt_rep;
        int nra;
        const TileLoc L = locate_cached(a, sm.rep, tile, TX, TY, TZ, dt_rep, nra);
        if (a.kick && L.rep != cur_rep) {
            // the block's tiles moved on to another replica: fold the max |v|
            // gathered so far into the previous one (block-uniform branch)
            if (cur_rep >= 0) flush_vmax<G::NT>(vmax2, sm.red, a.sc + cur_rep);
            cur_rep = L.rep;
            vmax2 = 0.0;
        }
        Vec4<T> *cur = sm.u + buf * 2 * G::PLANE;
        T U;
        if constexpr (DB) {
            const int nxt = tile + gridDim.x;
            if (nxt < a.ntiles) issue_tile<TX, TY, TZ, true>(a, sm.rep, sm.u + (buf ^ 1) * 2 * G::PLANE, nxt);
            cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();
            U = tile_umax<TX, TY, TZ>(cur, sm.red);
        } else {
            __syncthreads();
            U = stage_tile<T, TX, TY, TZ, true>(a, L, cur, sm.red);
        }
        const double hdt = 0.5 * dt_rep;
        const bool has_ra = a.tile_flag[tile] != 0 && nra > 0;
        const bool inbox = (L.c0x + lx < L.rd.nx) && (L.c0y + ly < L.rd.ny) && (L.c0z + lz < L.rd.nz);
        const Vec4<T> ui = cur[slot];
        const bool live = inbox && ui.x < (T)(0.5f * kVacant);
        Acc<T> fx, fy, fz;
        double ephi = 0.0;
        if (live) {
            const T lim = a.rc_lat + sqrt(ui.x * ui.x + ui.y * ui.y + ui.z * ui.z) + U;
            force_shells<T, 0, ENERGY>(a.sh, po, cur, slot, ui, lim * lim, a.S, seglo, nseg1, tab0, tab1, a.tab_phi, fx,
                                       fy, fz, ephi);
        }
        if (has_ra) {
            int pos = 0;
            const int sx = 2 * lx + p, sy = 2 * ly + p, sz = 2 * lz + p;
            while (true) {
                __syncthreads();
                const int cnt = stage_runaways<T, TX, TY, TZ, true>(a, L, tile, nra, pos, sm.rh, sm.ru, sm.st);
                if (cnt == 0) break;
                if (live) {
                    for (int j = 0; j < cnt; ++j) {
                        const Vec4<T> uj = sm.ru[j];
                        const RaPair<T> P = ra_pair<T>(a, L.rd, sm.rh[j], uj, ui, sx, sy, sz);
                        if (P.in) {
                            const Vec4<T> c0 = a.tab_d0[P.seg];
                            const Vec2<T> c1 = a.tab_d1[P.seg];
                            const T dfr = (c0.x * P.t + c0.y) * P.t + c0.z;
                            const T dph = (c0.w * P.t + c1.x) * P.t + c1.y;
                            const T coef = (ui.w + uj.w) * dfr + dph;
                            const T sc_ = P.floor_hit ? (T)0 : coef * P.rinv;
                            if (P.floor_hit) st |= kStRfloor;
                            fx.add(sc_ * P.rx);
                            fy.add(sc_ * P.ry);
                            fz.add(sc_ * P.rz);
                            if (ENERGY) {
                                const Vec4<T> cp = a.tab_phi[P.seg];
                                ephi += 0.5 * (double)(((cp.x * P.t + cp.y) * P.t + cp.z) * P.t + cp.w);
                            }
                        }
                    }
                }
                if (pos >= nra) break;
            }
        }
        if (live) {
            const long long sid =
                L.rd.site_base + (((long long)(L.c0z + lz) * L.rd.ny + (L.c0y + ly)) * L.rd.nx + (L.c0x + lx)) * 2 + p;
            T gx, gy, gz;
            if constexpr (sizeof(T) == 4) {
                gx = fx.value() * conv;
                gy = fy.value() * conv;
                gz = fz.value() * conv;
            } else {
                gx = fx.value() * a.acc_conv;
                gy = fy.value() * a.acc_conv;
                gz = fz.value() * a.acc_conv;
            }
            a.ax[sid] = gx;
            a.ay[sid] = gy;
            a.az[sid] = gz;
            if (!isfinite(gx) || !isfinite(gy) || !isfinite(gz)) st |= kStNonfinite;
            if (a.kick) {
                const double vx = fma(hdt, (double)gx, a.vx[sid]);
                const double vy = fma(hdt, (double)gy, a.vy[sid]);
                const double vz = fma(hdt, (double)gz, a.vz[sid]);
                a.vx[sid] = vx;
                a.vy[sid] = vy;
                a.vz[sid] = vz;
                const double v2 = vx * vx + vy * vy + vz * vz;
                vmax2 = v2 > vmax2 ? v2 : vmax2;
            }
            if (ENERGY) a.e_out[sid] += ephi;
        }
        if constexpr (DB) {
            buf ^= 1;
            __syncthreads();
        }
    }
    if (a.kick && cur_rep >= 0) flush_vmax<G::NT>(vmax2, sm.red, a.sc + cur_rep);
    if constexpr (DB) cp_async_wait<0>();
    if (st) atomicOr(&a.sc[0].status, st);
}

}  // namespace misa
