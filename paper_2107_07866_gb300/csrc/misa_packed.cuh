// misa_packed.cuh -- FP32 density and force passes with two sites per thread
// in packed FP32x2 arithmetic (Sec. 2.2 steps 1-5, Alg. 1 part 1).
//
// Blackwell issues add, multiply and fma on a pair of FP32 values in one
// instruction.  The gathers are issue-bound, so each thread owns two sites
// of a tile, (x, y, z) and (x, y, z + TZ/2), and evaluates every offset
// vector for both at once.  The tile plus its 2-cell halo is staged
// "folded": the shared-memory slot of cell (x, y, z') holds the sites at z'
// and z' + TZ/2 side by side, so that for any offset vector both of a
// thread's neighbours sit in one slot, already paired:
//   plane A: (ux_a, ux_b, uy_a, uy_b)   plane B: (uz_a, uz_b, F'_a, F'_b).
// Geometry and the spline argument run packed; the cubic of each site reads
// its own table segment and runs in scalar FMAs.
//
// The table window in shared memory ends with one all-zero segment; every
// segment index at or beyond rc (and any out-of-window index) is clamped to
// it, so candidates outside rc -- and vacant sites, whose displacement is
// the 1e4 sentinel -- contribute exactly zero without a mask.
//
// Sparse shells (|n|^2 > 12: at most a few of their candidates fall inside
// rc) are screened before any geometry: a pair can only be inside rc if
// |u_i| + |u_j| >= |n| - rc, and the density pass keeps |u_j|^2 in the
// fourth plane slot for that test.  It records, per site, a bit for every
// sparse candidate it found inside rc; the force pass, which sees the same
// FP32 displacements and makes the same decisions, evaluates only those.
//
// Per-site arithmetic is independent of the partner site and of the tile:
// a shell's sum is added (Kahan) only when it is non-zero, so shells that a
// wider or narrower visit bound includes or skips change nothing.
#pragma once

#include "misa_kernels.cuh"

namespace misa {

// ---------------------------------------------------------------------------
// packed FP32x2 operations (round to nearest, no contraction)
// ---------------------------------------------------------------------------

__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b as fma(b, -1, a): one rounding, the same as a subtraction
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 p_dup(float a) { return make_float2(a, a); }

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------------------
// folded tile geometry
// ---------------------------------------------------------------------------

template <int TX, int TY, int TZ>
struct PTile {
    static_assert(TZ % 2 == 0, "the packed tile folds z in halves");
    static constexpr int HZ = TZ / 2;
    static constexpr int SX = TX + 4, SY = TY + 4, SZ = HZ + 4;
    static constexpr int PLANE = SX * SY * SZ;    // folded slots per parity
    static constexpr int PER_PAR = TX * TY * HZ;  // threads per parity
    static constexpr int NT = 2 * PER_PAR;        // threads; two sites each
};

// shared-memory bytes of one staged tile (planes A and B, both parities)
__host__ __device__ inline size_t ptile_smem_bytes(int tx, int ty, int tz)
{
    return sizeof(float4) * 2 * 2 * (size_t)(tx + 4) * (ty + 4) * (tz / 2 + 4);
}

struct PackedSmem {
    RepCache *rep;
    float4 *tA;   // nbuf staged tiles, plane A then plane B each
    int4 *rh;
    Vec4<float> *ru;
    float *red;
    RaStage *st;
};

__host__ __device__ inline size_t packed_smem_bytes(size_t table_bytes, int tx, int ty, int tz, int nbuf)
{
    size_t off = (table_bytes + 255) & ~(size_t)255;
    off += sizeof(RepCache) * kRepSmem;
    off += ptile_smem_bytes(tx, ty, tz) * nbuf;
    off += sizeof(int4) * kRaChunk + sizeof(Vec4<float>) * kRaChunk + sizeof(float) * kRedFloats + sizeof(RaStage);
    return off;
}

template <int TX, int TY, int TZ>
__device__ __forceinline__ PackedSmem carve_p(unsigned char *smem, size_t off, int nbuf)
{
    PackedSmem g;
    off = (off + 255) & ~(size_t)255;
    g.rep = reinterpret_cast<RepCache *>(smem + off);
    off += sizeof(RepCache) * kRepSmem;
    g.tA = reinterpret_cast<float4 *>(smem + off);
    off += ptile_smem_bytes(TX, TY, TZ) * nbuf;
    g.rh = reinterpret_cast<int4 *>(smem + off);
    off += sizeof(int4) * kRaChunk;
    g.ru = reinterpret_cast<Vec4<float> *>(smem + off);
    off += sizeof(Vec4<float>) * kRaChunk;
    g.red = reinterpret_cast<float *>(smem + off);
    off += sizeof(float) * kRedFloats;
    g.st = reinterpret_cast<RaStage *>(smem + off);
    return g;
}

// block-wide max of a per-thread value (floats >= 0), all threads get it
template <int NT>
__device__ __forceinline__ float block_max(float m, float *sred)
{
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        float w = threadIdx.x < (NT >> 5) ? sred[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) w = fmaxf(w, __shfl_xor_sync(0xffffffffu, w, o));
        if (threadIdx.x == 0) sred[32] = w;
    }
    __syncthreads();
    return sred[32];
}

__device__ __forceinline__ float occ_u2(float x, float y, float z)
{
    return x < 0.5f * kVacant ? x * x + y * y + z * z : 0.f;
}

// global site ids of folded slot (p, x, y, z') of the tile at L
template <int TX, int TY, int TZ>
__device__ __forceinline__ void slot_sites(const TileLoc &L, int q, int &p, int &r, long long &sa, long long &sb)
{
    using G = PTile<TX, TY, TZ>;
    p = q & 1;
    r = q >> 1;
    const int x = r % G::SX;
    const int yz = r / G::SX;
    const int y = yz % G::SY;
    const int z = yz / G::SY;
    const int gx = wrap_cell(L.c0x - 2 + x, L.rd.nx);
    const int gy = wrap_cell(L.c0y - 2 + y, L.rd.ny);
    const int gza = wrap_cell(L.c0z - 2 + z, L.rd.nz);
    const int gzb = wrap_cell(L.c0z - 2 + z + G::HZ, L.rd.nz);
    const long long row = ((long long)gy * L.rd.nx + gx) * 2 + p;
    const long long zs = (long long)L.rd.ny * L.rd.nx * 2;
    sa = L.rd.site_base + gza * zs + row;
    sb = L.rd.site_base + gzb * zs + row;
}

// Synchronous staging of the folded tile + halo.  Returns max |u| over the
// occupied staged sites (lattice units, rounded up by one FP32 ulp).
template <int TX, int TY, int TZ, bool WITH_FP>
__device__ __forceinline__ float stage_tile_p(const GatherArgs<float> &a, const TileLoc &L, float4 *sA, float *sred)
{
    using G = PTile<TX, TY, TZ>;
    float4 *sB = sA + 2 * G::PLANE;
    float umax2 = 0.f;
    for (int q = threadIdx.x; q < 2 * G::PLANE; q += G::NT) {
        int p, r;
        long long sa, sb;
        slot_sites<TX, TY, TZ>(L, q, p, r, sa, sb);
        const float xa = a.ux[sa], xb = a.ux[sb];
        const float ya = a.uy[sa], yb = a.uy[sb];
        const float za = a.uz[sa], zb = a.uz[sb];
        // force pass: F' of both sites; density pass: |u|^2 of both sites
        const float fa = WITH_FP ? a.fp[sa] : xa * xa + ya * ya + za * za;
        const float fb = WITH_FP ? a.fp[sb] : xb * xb + yb * yb + zb * zb;
        umax2 = fmaxf(umax2, fmaxf(occ_u2(xa, ya, za), occ_u2(xb, yb, zb)));
        sA[p * G::PLANE + r] = make_float4(xa, xb, ya, yb);
        sB[p * G::PLANE + r] = make_float4(za, zb, fa, fb);
    }
    return sqrtf(block_max<G::NT>(umax2, sred)) * 1.000001f;
}

// Asynchronous staging (cp.async, 4-byte copies into the paired positions).
template <int TX, int TY, int TZ, bool WITH_FP>
__device__ __forceinline__ void issue_tile_p(const GatherArgs<float> &a, const RepCache *rc, float4 *sA, int tile)
{
    using G = PTile<TX, TY, TZ>;
    float4 *sB = sA + 2 * G::PLANE;
    double dt_;
    int nra_;
    const TileLoc L = locate_cached(a, rc, tile, TX, TY, TZ, dt_, nra_);
    for (int q = threadIdx.x; q < 2 * G::PLANE; q += G::NT) {
        int p, r;
        long long sa, sb;
        slot_sites<TX, TY, TZ>(L, q, p, r, sa, sb);
        float4 *A = sA + p * G::PLANE + r;
        float4 *B = sB + p * G::PLANE + r;
        cp_async4(&A->x, a.ux + sa);
        cp_async4(&A->y, a.ux + sb);
        cp_async4(&A->z, a.uy + sa);
        cp_async4(&A->w, a.uy + sb);
        cp_async4(&B->x, a.uz + sa);
        cp_async4(&B->y, a.uz + sb);
        if (WITH_FP) {
            cp_async4(&B->z, a.fp + sa);
            cp_async4(&B->w, a.fp + sb);
        }
    }
}

// Max |u| over the occupied slots of a staged tile, block-wide; with
// WRITE_U2 (density pass) each slot's |u|^2 pair goes to plane B's zw.
template <int TX, int TY, int TZ, bool WRITE_U2>
__device__ __forceinline__ float tile_umax_p(float4 *sA, float *sred)
{
    using G = PTile<TX, TY, TZ>;
    float4 *sB = sA + 2 * G::PLANE;
    float umax2 = 0.f;
    for (int q = threadIdx.x; q < 2 * G::PLANE; q += G::NT) {
        const float4 A = sA[q];
        float4 B = sB[q];
        const float ua = A.x * A.x + A.z * A.z + B.x * B.x, ub = A.y * A.y + A.w * A.w + B.y * B.y;
        umax2 = fmaxf(umax2, fmaxf(A.x < 0.5f * kVacant ? ua : 0.f, A.y < 0.5f * kVacant ? ub : 0.f));
        if (WRITE_U2) {
            B.z = ua;
            B.w = ub;
            sB[q] = B;
        }
    }
    return sqrtf(block_max<G::NT>(umax2, sred)) * 1.000001f;
}

// ---------------------------------------------------------------------------
// packed shell loops
// ---------------------------------------------------------------------------

struct PShell {
    float2 n2, nrm, xfrac;
    float thr;
    int xo;  // segment offset in the shared-memory window, incl. the rounding trick
};

template <int SH>
__device__ __forceinline__ PShell pshell(const ShellInfo &sh, int seg_lo)
{
    PShell r;
    constexpr int N2 = kLVec.shell_n2[SH];
    r.n2 = p_dup((float)N2);
    r.nrm = p_dup(sh.nrm[SH]);
    r.xfrac = p_dup(sh.xfrac[SH]);
    r.thr = sh.thr[SH];
    r.xo = sh.xoff[SH] - seg_lo;
    return r;
}

// Spline argument of both pairs (see shell_arg): segment indices into the
// window (clamped to the zero segment nwin), t, and 1/r.
__device__ __forceinline__ void arg_p(const PShell &sh, float2 q, float2 S2, unsigned nwin, float2 &t, float2 &rs,
                                      int &ia, int &ib)
{
    const float2 r2 = p_add(sh.n2, q);
    rs = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
    const float2 r = p_mul(r2, rs);
    const float2 den = p_add(r, sh.nrm);
    const float2 dr = p_mul(q, make_float2(rcp_approx(den.x), rcp_approx(den.y)));
    const float2 x = p_fma(dr, S2, sh.xfrac);
    const float2 y = p_add(p_add(x, p_dup(-0.5f)), p_dup(12582912.0f));
    const float2 fl = p_add(y, p_dup(-12582912.0f));
    t = p_sub(x, fl);
    ia = (int)min((unsigned)(__float_as_int(y.x) + sh.xo), nwin);
    ib = (int)min((unsigned)(__float_as_int(y.y) + sh.xo), nwin);
}

__device__ __forceinline__ float cubic(const float4 c, float t) { return fmaf(fmaf(fmaf(c.x, t, c.y), t, c.z), t, c.w); }

struct PairSites {
    float2 ux, uy, uz, fp;  // the thread's two sites
};

// first sparse shell and its first candidate
constexpr int first_sparse_shell()
{
    int s = 0;
    while (s < kLVec.nshell && kLVec.shell_n2[s] <= 12) ++s;
    return s;
}
constexpr int kSparseShell = first_sparse_shell();
constexpr int kSparseK0 = kLVec.shell_begin[kSparseShell];

// both pairs of candidate k: d = u_j - u_i, 2n and q = (2n + d).d
struct PGeom {
    float2 dx, dy, dz, nx2, ny2, nz2, q;
};

__device__ __forceinline__ PGeom pair_geom(const float4 o0, const float4 o1, const float4 A, const float4 B,
                                           const PairSites &ui)
{
    PGeom g;
    g.dx = p_sub(make_float2(A.x, A.y), ui.ux);
    g.dy = p_sub(make_float2(A.z, A.w), ui.uy);
    g.dz = p_sub(make_float2(B.x, B.y), ui.uz);
    g.nx2 = make_float2(o0.x, o0.y);
    g.ny2 = make_float2(o0.z, o0.w);
    g.nz2 = make_float2(o1.x, o1.y);
    g.q = p_fma(p_add(g.dz, g.nz2), g.dz, p_fma(p_add(g.dy, g.ny2), g.dy, p_mul(p_add(g.dx, g.nx2), g.dx)));
    return g;
}

__device__ __forceinline__ void kahan_nz(Acc<float> &acc, float v)
{
    if (v != 0.f) acc.add(v);
}

// Screening bound of a sparse shell for one site: a neighbour j can only be
// inside rc if |u_j|^2 >= thr (lattice units; -1: always).  A margin of
// 1e-4 lattice units keeps every pair the FP32 geometry would place inside rc.
__device__ __forceinline__ float screen_thr(float nrm, float rc_lat, float ui_norm, bool need)
{
    if (!need) return 3.0e38f;
    const float gap = nrm - rc_lat - 1.0e-4f - ui_norm;
    return gap > 0.f ? gap * gap * 0.99999f : -1.f;
}

// Table reads of the two sites take two paths of the L1 unit that run side
// by side: site a from shared memory, site b through the texture path (a
// texture object over the global table; shared memory when there is none).
__device__ __forceinline__ float4 tab_b(const float4 *__restrict__ tab, unsigned long long tex, int seg_lo, int i)
{
    if (tex) return tex1Dfetch<float4>((cudaTextureObject_t)tex, seg_lo + i);
    return tab[i];
}

template <int SH>
__device__ __forceinline__ void density_shells_p(const ShellInfo &shc, int seg_lo, const float4 *__restrict__ po,
                                                 const float4 *__restrict__ sA, const float4 *__restrict__ sB, int slot,
                                                 const PairSites &ui, float2 unorm, float rc_lat, float2 lim2, float2 S2,
                                                 unsigned nwin, const float4 *__restrict__ tab, unsigned long long texf,
                                                 Acc<float> &ra, Acc<float> &rb, unsigned long long &ma,
                                                 unsigned long long &mb)
{
    if constexpr (SH < kLVec.nshell) {
        constexpr int KB = kLVec.shell_begin[SH], KE = kLVec.shell_begin[SH + 1];
        constexpr int N2 = kLVec.shell_n2[SH];
        constexpr bool dense = SH < kSparseShell;
        const bool na = (float)N2 <= lim2.x, nb = (float)N2 <= lim2.y;
        if (SH >= shc.nshell || !(na || nb)) return;
        const PShell sh = pshell<SH>(shc, seg_lo);
        float2 part = make_float2(0.f, 0.f);
        if constexpr (dense) {
#pragma unroll 2
            for (int k = KB; k < KE; ++k) {
                const float4 o0 = po[2 * k], o1 = po[2 * k + 1];
                const int D = __float_as_int(o1.z);
                const PGeom g = pair_geom(o0, o1, sA[slot + D], sB[slot + D], ui);
                float2 t, rs;
                int ia, ib;
                arg_p(sh, g.q, S2, nwin, t, rs, ia, ib);
                part = p_add(part, make_float2(cubic(tab[ia], t.x), cubic(tab_b(tab, texf, seg_lo, ib), t.y)));
            }
        } else {
            const float ta = screen_thr(shc.nrm[SH], rc_lat, unorm.x, na);
            const float tb = screen_thr(shc.nrm[SH], rc_lat, unorm.y, nb);
            for (int k = KB; k < KE; ++k) {
                const float4 o1 = po[2 * k + 1];
                const int D = __float_as_int(o1.z);
                const float4 B = sB[slot + D];  // zw: |u_j|^2 of both neighbours
                if (B.z >= ta || B.w >= tb) {
                    const PGeom g = pair_geom(po[2 * k], o1, sA[slot + D], B, ui);
                    float2 t, rs;
                    int ia, ib;
                    arg_p(sh, g.q, S2, nwin, t, rs, ia, ib);
                    part = p_add(part, make_float2(cubic(tab[ia], t.x), cubic(tab_b(tab, texf, seg_lo, ib), t.y)));
                    const int bi = k - kSparseK0;
                    if (bi < 64) {  // configurations with more sparse candidates run unmasked
                        const unsigned long long bit = 1ull << bi;
                        if (ia < (int)nwin) ma |= bit;
                        if (ib < (int)nwin) mb |= bit;
                    }
                }
            }
        }
        kahan_nz(ra, part.x);
        kahan_nz(rb, part.y);
        density_shells_p<SH + 1>(shc, seg_lo, po, sA, sB, slot, ui, unorm, rc_lat, lim2, S2, nwin, tab, texf, ra, rb, ma,
                                 mb);
    }
}

struct ForceTex {
    unsigned long long d0, d1;
};

// one candidate of the force pass for both sites, accumulated into p*
template <bool ENERGY>
__device__ __forceinline__ void force_pair_p(const PShell &sh, const PGeom &g, const float4 B, const PairSites &ui,
                                             float2 S2, unsigned nwin, int seg_lo, const float4 *__restrict__ tab0,
                                             const float2 *__restrict__ tab1, const ForceTex &tx,
                                             const Vec4<float> *__restrict__ gphi, float2 &px, float2 &py, float2 &pz,
                                             double &ea, double &eb)
{
    float2 t, rs;
    int ia, ib;
    arg_p(sh, g.q, S2, nwin, t, rs, ia, ib);
    // f' and the t^2 coefficient of phi' from shared memory, the rest of phi'
    // through the texture path (the global table, whose last entry is the
    // zero segment, without texture objects)
    const float4 ca = tab0[ia], cb = tab0[ib];
    float2 da, db;
    if (tx.d1) {
        da = tex1Dfetch<float2>((cudaTextureObject_t)tx.d1, seg_lo + ia);
        db = tex1Dfetch<float2>((cudaTextureObject_t)tx.d1, seg_lo + ib);
    } else {
        da = tab1[seg_lo + ia];
        db = tab1[seg_lo + ib];
    }
    const float2 dfr = make_float2(fmaf(fmaf(ca.x, t.x, ca.y), t.x, ca.z), fmaf(fmaf(cb.x, t.y, cb.y), t.y, cb.z));
    const float2 dph = make_float2(fmaf(fmaf(ca.w, t.x, da.x), t.x, da.y), fmaf(fmaf(cb.w, t.y, db.x), t.y, db.y));
    const float2 sc = p_mul(p_fma(p_add(ui.fp, make_float2(B.z, B.w)), dfr, dph), rs);
    // r_ij = n + d, with n = (2n)/2 exactly
    px = p_fma(sc, p_fma(p_dup(0.5f), g.nx2, g.dx), px);
    py = p_fma(sc, p_fma(p_dup(0.5f), g.ny2, g.dy), py);
    pz = p_fma(sc, p_fma(p_dup(0.5f), g.nz2, g.dz), pz);
    if (ENERGY) {
        const int ua = (int)nwin;
        if (ia < ua) ea += 0.5 * (double)cubic(*reinterpret_cast<const float4 *>(&gphi[seg_lo + ia]), t.x);
        if (ib < ua) eb += 0.5 * (double)cubic(*reinterpret_cast<const float4 *>(&gphi[seg_lo + ib]), t.y);
    }
}

__device__ __forceinline__ void kahan3_nz(Acc<float> (&f)[3], float x, float y, float z)
{
    kahan_nz(f[0], x);
    kahan_nz(f[1], y);
    kahan_nz(f[2], z);
}

// Shells SH.. of the force pass.  Dense shells evaluate every candidate;
// sparse shells evaluate the candidates set in msk (the union of both
// sites' density-pass bits) or, without masks, every candidate that the
// visit bound admits.
template <int SH, bool ENERGY>
__device__ __forceinline__ void force_shells_p(const ShellInfo &shc, int seg_lo, const float4 *__restrict__ po,
                                               const float4 *__restrict__ sA, const float4 *__restrict__ sB, int slot,
                                               const PairSites &ui, float2 lim2, float2 S2, unsigned nwin,
                                               const float4 *__restrict__ tab0, const float2 *__restrict__ tab1,
                                               const ForceTex &tx, const Vec4<float> *__restrict__ gphi, bool use_mask,
                                               unsigned long long msk, Acc<float> (&fa)[3], Acc<float> (&fb)[3],
                                               double &ea, double &eb)
{
    if constexpr (SH < kLVec.nshell) {
        constexpr int KB = kLVec.shell_begin[SH], KE = kLVec.shell_begin[SH + 1];
        constexpr int N2 = kLVec.shell_n2[SH];
        constexpr bool dense = SH < kSparseShell;
        const bool na = (float)N2 <= lim2.x, nb = (float)N2 <= lim2.y;
        if (SH >= shc.nshell || !(na || nb)) return;
        const PShell sh = pshell<SH>(shc, seg_lo);
        float2 px = make_float2(0.f, 0.f), py = px, pz = px;
        if (dense || !use_mask) {
#pragma unroll 2
            for (int k = KB; k < KE; ++k) {
                const float4 o0 = po[2 * k], o1 = po[2 * k + 1];
                const int D = __float_as_int(o1.z);
                const float4 B = sB[slot + D];
                const PGeom g = pair_geom(o0, o1, sA[slot + D], B, ui);
                if (dense || g.q.x < sh.thr || g.q.y < sh.thr)
                    force_pair_p<ENERGY>(sh, g, B, ui, S2, nwin, seg_lo, tab0, tab1, tx, gphi, px, py, pz, ea, eb);
            }
        } else {
            unsigned long long sub = (msk >> (KB - kSparseK0)) & ((1ull << (KE - KB)) - 1ull);
            while (sub) {
                const int k = KB + __ffsll((long long)sub) - 1;
                sub &= sub - 1ull;
                const float4 o0 = po[2 * k], o1 = po[2 * k + 1];
                const int D = __float_as_int(o1.z);
                const float4 B = sB[slot + D];
                const PGeom g = pair_geom(o0, o1, sA[slot + D], B, ui);
                force_pair_p<ENERGY>(sh, g, B, ui, S2, nwin, seg_lo, tab0, tab1, tx, gphi, px, py, pz, ea, eb);
            }
        }
        kahan3_nz(fa, px.x, py.x, pz.x);
        kahan3_nz(fb, px.y, py.y, pz.y);
        force_shells_p<SH + 1, ENERGY>(shc, seg_lo, po, sA, sB, slot, ui, lim2, S2, nwin, tab0, tab1, tx, gphi, use_mask,
                                       msk, fa, fb, ea, eb);
    }
}

// ---------------------------------------------------------------------------
// run-away pairs of one site (scalar, as in the one-site-per-thread kernels)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void ra_density_site(const GatherArgs<float> &a, const TileLoc &L, int cnt, const int4 *rh,
                                                const Vec4<float> *ru, const Vec4<float> &ui, int sx, int sy, int sz,
                                                Acc<float> &rho, unsigned &st)
{
    for (int j = 0; j < cnt; ++j) {
        const RaPair<float> P = ra_pair<float>(a, L.rd, rh[j], ru[j], ui, sx, sy, sz);
        if (P.in) {
            if (P.floor_hit) st |= kStRfloor;
            const Vec4<float> c = a.tab_f[P.seg];
            rho.add(((c.x * P.t + c.y) * P.t + c.z) * P.t + c.w);
        }
    }
}

template <bool ENERGY>
__device__ __forceinline__ void ra_force_site(const GatherArgs<float> &a, const TileLoc &L, int cnt, const int4 *rh,
                                              const Vec4<float> *ru, const Vec4<float> &ui, int sx, int sy, int sz,
                                              Acc<float> (&f)[3], double &e, unsigned &st)
{
    for (int j = 0; j < cnt; ++j) {
        const Vec4<float> uj = ru[j];
        const RaPair<float> P = ra_pair<float>(a, L.rd, rh[j], uj, ui, sx, sy, sz);
        if (P.in) {
            const Vec4<float> c0 = a.tab_d0[P.seg];
            const Vec2<float> c1 = a.tab_d1[P.seg];
            const float dfr = (c0.x * P.t + c0.y) * P.t + c0.z;
            const float dph = (c0.w * P.t + c1.x) * P.t + c1.y;
            const float coef = (ui.w + uj.w) * dfr + dph;
            const float sc_ = P.floor_hit ? 0.f : coef * P.rinv;
            if (P.floor_hit) st |= kStRfloor;
            f[0].add(sc_ * P.rx);
            f[1].add(sc_ * P.ry);
            f[2].add(sc_ * P.rz);
            if (ENERGY) {
                const Vec4<float> cp = a.tab_phi[P.seg];
                e += 0.5 * (double)(((cp.x * P.t + cp.y) * P.t + cp.z) * P.t + cp.w);
            }
        }
    }
}

// This thread's two sites in the tile: parity p, local cell (lx, ly, lz) and
// (lx, ly, lz + TZ/2).
template <int TX, int TY, int TZ>
struct PThread {
    int p, lx, ly, lz, slot;
    __device__ __forceinline__ PThread()
    {
        using G = PTile<TX, TY, TZ>;
        const int q = threadIdx.x;
        p = q / G::PER_PAR;
        const int rr = q % G::PER_PAR;
        lx = rr % TX;
        ly = (rr / TX) % TY;
        lz = rr / (TX * TY);
        slot = p * G::PLANE + ((lz + 2) * G::SY + (ly + 2)) * G::SX + (lx + 2);
    }
};

__device__ __forceinline__ long long site_of(const TileLoc &L, int lx, int ly, int lz, int p)
{
    return L.rd.site_base + (((long long)(L.c0z + lz) * L.rd.ny + (L.c0y + ly)) * L.rd.nx + (L.c0x + lx)) * 2 + p;
}

// ---------------------------------------------------------------------------
// density pass: rho_i, F'(rho_i)
// ---------------------------------------------------------------------------

template <int TX, int TY, int TZ, bool ENERGY, bool DB>
__global__ void __launch_bounds__(TX *TY *TZ, 1) k_density_p(const __grid_constant__ GatherArgs<float> a)
{
    using G = PTile<TX, TY, TZ>;
    extern __shared__ __align__(32) unsigned char smem[];
    const int nwin = a.nseg - a.seg_lo;
    float4 *tab = reinterpret_cast<float4 *>(smem);
    for (int k = threadIdx.x; k <= nwin; k += G::NT) {
        const Vec4<float> c = k < nwin ? a.tab_f[a.seg_lo + k] : Vec4<float>{0.f, 0.f, 0.f, 0.f};
        tab[k] = make_float4(c.x, c.y, c.z, c.w);
    }
    const PackedSmem sm = carve_p<TX, TY, TZ>(smem, sizeof(float4) * (size_t)(nwin + 1), DB ? 2 : 1);
    fill_rep_cache<float>(a, sm.rep);
    __syncthreads();

    const PThread<TX, TY, TZ> th;
    // offset records read from the kernel parameters (constant bank): warp-
    // uniform, so they stay off the shared-memory pipe
    const float4 *po = &a.offp[th.p][0][0];
    const float2 S2 = p_dup(a.S);
    unsigned st = 0;
    int buf = 0;
    // double-buffered: the next tile streams in (cp.async) during the whole
    // tile; single buffer: plain loads at the top of each tile
    if constexpr (DB) {
        if ((int)blockIdx.x < a.ntiles) issue_tile_p<TX, TY, TZ, false>(a, sm.rep, sm.tA, blockIdx.x);
        cp_async_commit();
    }
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        double dt_rep;
        int nra;
        const TileLoc L = locate_cached(a, sm.rep, tile, TX, TY, TZ, dt_rep, nra);
        float4 *cA = sm.tA + buf * 4 * G::PLANE;
        const float4 *cB = cA + 2 * G::PLANE;
        float U;
        if constexpr (DB) {
            const int nxt = tile + gridDim.x;
            if (nxt < a.ntiles) issue_tile_p<TX, TY, TZ, false>(a, sm.rep, sm.tA + (buf ^ 1) * 4 * G::PLANE, nxt);
            cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();
            U = tile_umax_p<TX, TY, TZ, true>(cA, sm.red);
        } else {
            __syncthreads();
            U = stage_tile_p<TX, TY, TZ, false>(a, L, cA, sm.red);
        }
        const bool has_ra = a.tile_flag[tile] != 0 && nra > 0;
        const bool in_xy = (L.c0x + th.lx < L.rd.nx) && (L.c0y + th.ly < L.rd.ny);
        const bool in_a = in_xy && (L.c0z + th.lz < L.rd.nz);
        const bool in_b = in_xy && (L.c0z + th.lz + G::HZ < L.rd.nz);
        const float4 A = cA[th.slot], B = cB[th.slot];
        PairSites ui;
        ui.ux = make_float2(A.x, A.y);
        ui.uy = make_float2(A.z, A.w);
        ui.uz = make_float2(B.x, B.y);
        ui.fp = make_float2(0.f, 0.f);
        const bool live_a = in_a && A.x < 0.5f * kVacant;
        const bool live_b = in_b && A.y < 0.5f * kVacant;
        Acc<float> ra, rb;
        unsigned long long ma = 0, mb = 0;
        if (live_a || live_b) {
            const float2 un = make_float2(sqrtf(A.x * A.x + A.z * A.z + B.x * B.x), sqrtf(A.y * A.y + A.w * A.w + B.y * B.y));
            const float la = a.rc_lat + un.x + U, lb = a.rc_lat + un.y + U;
            const float2 lim2 = make_float2(live_a ? la * la : -1.f, live_b ? lb * lb : -1.f);
            density_shells_p<0>(a.sh, a.seg_lo, po, cA, cB, th.slot, ui, un, a.rc_lat, lim2, S2, (unsigned)nwin, tab,
                                a.tex_f, ra, rb, ma, mb);
        }
        if (has_ra) {
            int pos = 0;
            const int sx = 2 * th.lx + th.p, sy = 2 * th.ly + th.p;
            const int sza = 2 * th.lz + th.p, szb = 2 * (th.lz + G::HZ) + th.p;
            const Vec4<float> ua{A.x, A.z, B.x, 0.f}, ub{A.y, A.w, B.y, 0.f};
            while (true) {
                __syncthreads();
                const int cnt = stage_runaways<float, TX, TY, TZ, false>(a, L, tile, nra, pos, sm.rh, sm.ru, sm.st);
                if (cnt == 0) break;
                if (live_a) ra_density_site(a, L, cnt, sm.rh, sm.ru, ua, sx, sy, sza, ra, st);
                if (live_b) ra_density_site(a, L, cnt, sm.rh, sm.ru, ub, sx, sy, szb, rb, st);
                if (pos >= nra) break;
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const bool in = h ? in_b : in_a;
            if (!in) continue;
            const long long sid = site_of(L, th.lx, th.ly, th.lz + h * G::HZ, th.p);
            if (!(h ? live_b : live_a)) {
                a.fp_out[sid] = 0.f;  // vacant: F' = 0 keeps every product with it finite
                continue;
            }
            if (a.mask_ok) a.bmask[sid] = h ? mb : ma;
            const float rh = (h ? rb : ra).value();
            float dF;
            const float Fv = embed<float>(a.tab_F, a.nseg, a.Srho, a.rho_max, rh, dF, st);
            a.fp_out[sid] = dF;
            if (ENERGY) {
                a.rho_out[sid] = rh;
                a.e_out[sid] = (double)Fv;
            }
        }
        if constexpr (DB) {
            buf ^= 1;
            __syncthreads();  // every read of the current buffer is done before it is refilled
        }
    }
    if constexpr (DB) cp_async_wait<0>();
    if (st) atomicOr(&a.sc[0].status, st);
}

// ---------------------------------------------------------------------------
// force pass + closing half kick
// ---------------------------------------------------------------------------

// The tile loop overlaps the staging of the next tile with the FP64 kick
// epilogue of the current one: once every thread has read the staged tile,
// the next tile's copies are issued (cp.async) and fly while the kick runs.
template <int TX, int TY, int TZ, bool ENERGY>
__global__ void __launch_bounds__(TX *TY *TZ, 1) k_force_p(const __grid_constant__ GatherArgs<float> a)
{
    using G = PTile<TX, TY, TZ>;
    extern __shared__ __align__(32) unsigned char smem[];
    const int nwin = a.nseg - a.seg_lo;
    float4 *tab0 = reinterpret_cast<float4 *>(smem);
    for (int k = threadIdx.x; k <= nwin; k += G::NT) {
        const Vec4<float> c0 = k < nwin ? a.tab_d0[a.seg_lo + k] : Vec4<float>{0.f, 0.f, 0.f, 0.f};
        tab0[k] = make_float4(c0.x, c0.y, c0.z, c0.w);
    }
    const PackedSmem sm = carve_p<TX, TY, TZ>(smem, sizeof(float4) * (size_t)(nwin + 1), 1);
    fill_rep_cache<float>(a, sm.rep);
    __syncthreads();

    const PThread<TX, TY, TZ> th;
    // offset records read from the kernel parameters (constant bank): warp-
    // uniform, so they stay off the shared-memory pipe
    const float4 *po = &a.offp[th.p][0][0];
    const float2 S2 = p_dup(a.S);
    const float conv = (float)a.acc_conv;
    unsigned st = 0;
    int cur_rep = -1;
    unsigned long long vmax2 = 0;  // bits of a non-negative double: integer order = value order
    float4 *cA = sm.tA;
    const float4 *cB = cA + 2 * G::PLANE;
    if ((int)blockIdx.x < a.ntiles) issue_tile_p<TX, TY, TZ, true>(a, sm.rep, cA, blockIdx.x);
    cp_async_commit();
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        double dt_rep;
        int nra;
        const TileLoc L = locate_cached(a, sm.rep, tile, TX, TY, TZ, dt_rep, nra);
        if (a.kick && L.rep != cur_rep) {
            if (cur_rep >= 0) flush_vmax<G::NT>(__longlong_as_double((long long)vmax2), sm.red, a.sc + cur_rep);
            cur_rep = L.rep;
            vmax2 = 0;
        }
        cp_async_wait<0>();
        __syncthreads();
        const float U = tile_umax_p<TX, TY, TZ, false>(cA, sm.red);
        const double hdt = 0.5 * dt_rep;
        const bool has_ra = a.tile_flag[tile] != 0 && nra > 0;
        const bool in_xy = (L.c0x + th.lx < L.rd.nx) && (L.c0y + th.ly < L.rd.ny);
        const bool in_a = in_xy && (L.c0z + th.lz < L.rd.nz);
        const bool in_b = in_xy && (L.c0z + th.lz + G::HZ < L.rd.nz);
        const float4 A = cA[th.slot], B = cB[th.slot];
        PairSites ui;
        ui.ux = make_float2(A.x, A.y);
        ui.uy = make_float2(A.z, A.w);
        ui.uz = make_float2(B.x, B.y);
        ui.fp = make_float2(B.z, B.w);
        const bool live_a = in_a && A.x < 0.5f * kVacant;
        const bool live_b = in_b && A.y < 0.5f * kVacant;
        Acc<float> fa[3], fb[3];
        double ea = 0.0, eb = 0.0;
        if (live_a || live_b) {
            const float la = a.rc_lat + sqrtf(A.x * A.x + A.z * A.z + B.x * B.x) + U;
            const float lb = a.rc_lat + sqrtf(A.y * A.y + A.w * A.w + B.y * B.y) + U;
            const float2 lim2 = make_float2(live_a ? la * la : -1.f, live_b ? lb * lb : -1.f);
            unsigned long long msk = 0;
            if (a.mask_ok) {
                if (live_a) msk |= a.bmask[site_of(L, th.lx, th.ly, th.lz, th.p)];
                if (live_b) msk |= a.bmask[site_of(L, th.lx, th.ly, th.lz + G::HZ, th.p)];
            }
            const ForceTex tx{a.tex_d0, a.tex_d1};
            const float2 *t1 = reinterpret_cast<const float2 *>(a.tab_d1);
            force_shells_p<0, ENERGY>(a.sh, a.seg_lo, po, cA, cB, th.slot, ui, lim2, S2, (unsigned)nwin, tab0, t1, tx,
                                      a.tab_phi, a.mask_ok != 0, msk, fa, fb, ea, eb);
        }
        if (has_ra) {
            int pos = 0;
            const int sx = 2 * th.lx + th.p, sy = 2 * th.ly + th.p;
            const int sza = 2 * th.lz + th.p, szb = 2 * (th.lz + G::HZ) + th.p;
            const Vec4<float> ua{A.x, A.z, B.x, B.z}, ub{A.y, A.w, B.y, B.w};
            while (true) {
                __syncthreads();
                const int cnt = stage_runaways<float, TX, TY, TZ, true>(a, L, tile, nra, pos, sm.rh, sm.ru, sm.st);
                if (cnt == 0) break;
                if (live_a) ra_force_site<ENERGY>(a, L, cnt, sm.rh, sm.ru, ua, sx, sy, sza, fa, ea, st);
                if (live_b) ra_force_site<ENERGY>(a, L, cnt, sm.rh, sm.ru, ub, sx, sy, szb, fb, eb, st);
                if (pos >= nra) break;
            }
        }
        // every read of the staged tile is done: stage the next one during the kick
        __syncthreads();
        const int nxt = tile + gridDim.x;
        if (nxt < a.ntiles) issue_tile_p<TX, TY, TZ, true>(a, sm.rep, cA, nxt);
        cp_async_commit();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!(h ? live_b : live_a)) continue;
            const long long sid = site_of(L, th.lx, th.ly, th.lz + h * G::HZ, th.p);
            const Acc<float> *f = h ? fb : fa;
            const float gx = f[0].value() * conv, gy = f[1].value() * conv, gz = f[2].value() * conv;
            a.ax[sid] = gx;
            a.ay[sid] = gy;
            a.az[sid] = gz;
            if (!isfinite(gx) || !isfinite(gy) || !isfinite(gz)) st |= kStNonfinite;
            if (a.kick) {
                const double vx = fma(hdt, f2d_bits(gx), a.vx[sid]);
                const double vy = fma(hdt, f2d_bits(gy), a.vy[sid]);
                const double vz = fma(hdt, f2d_bits(gz), a.vz[sid]);
                a.vx[sid] = vx;
                a.vy[sid] = vy;
                a.vz[sid] = vz;
                const double v2 = vx * vx + vy * vy + vz * vz;
                const unsigned long long b = (unsigned long long)__double_as_longlong(v2);
                vmax2 = b > vmax2 ? b : vmax2;
            }
            if (ENERGY) a.e_out[sid] += h ? eb : ea;
        }
    }
    cp_async_wait<0>();
    if (a.kick && cur_rep >= 0) flush_vmax<G::NT>(__longlong_as_double((long long)vmax2), sm.red, a.sc + cur_rep);
    if (st) atomicOr(&a.sc[0].status, st);
}

}  // namespace misa
