// misa_alloy_packed.cuh -- FP32 density and force passes for alloys in the
// packed two-sites-per-thread form of the single-type gathers (Sec. 2.2
// steps 1-5 with atom types: Eq. eam_base and Eq. eam_force_ij).
//
// Tile staging, offset index, shell loops, sparse-shell screening and masks
// are those of misa_packed.cuh.  A third staged plane holds the species of
// both sites of every folded slot (species a | species b << 8; a vacant site
// reads species 0 and adds zero through its displacement sentinel).  The
// tables of an alloy (a density and an embedding function per species, a
// pair function per unordered species pair) do not all fit beside the
// staged tile in shared memory.  The density pass keeps the window
// (segments an array-array pair can reach) of the dominant species m's
// density function there, as the single-type pass does, and reads the other
// species' through the texture path; the force pass reads every table
// through the texture path (its texture latency is not hidden better by a
// window: a warp whose lanes mix species waits for the fetch either way).
// Texture reads are indexed by species and segment over the whole table;
// the last segment of every table is all zero and indices at or beyond rc
// clamp to it (the window's zero entry is the same segment).
//
// Density: rho_i = sum_j rho_{t_j}(r_ij), F'_i from the embedding function
// of t_i.  Force: [F'_i rho'_{t_j}(r) + F'_j rho'_{t_i}(r) + phi'_{t_i t_j}(r)]
// along r_hat, then the closing half kick as in the single-type pass.
#pragma once

#include "misa_alloy.cuh"
#include "misa_packed.cuh"

namespace misa {

// bytes of the species plane of a staged tile (one 16-bit pair per folded slot)
__host__ __device__ inline size_t ptype_smem_bytes(int tx, int ty, int tz)
{
    const size_t plane = (size_t)(tx + 4) * (ty + 4) * (tz / 2 + 4);
    return (sizeof(unsigned short) * 2 * plane + 255) & ~(size_t)255;
}

// shared-memory bytes of the dominant species' density window (nwin
// segments plus the zero one); the force pass holds no window
__host__ __device__ inline size_t alloy_window_bytes(bool force, int nwin)
{
    return force ? 0 : sizeof(float4) * (size_t)(nwin + 1);
}

// shared memory of the alloy passes: the window, the replica cache, the
// staged tile, the run-away chunk, then the species plane
__host__ __device__ inline size_t alloy_smem_bytes(bool force, int nwin, int tx, int ty, int tz)
{
    return ((packed_smem_bytes(alloy_window_bytes(force, nwin), tx, ty, tz, 1) + 255) & ~(size_t)255) +
           ptype_smem_bytes(tx, ty, tz);
}

__device__ __forceinline__ unsigned short site_species(const GatherArgs<float> &a, long long s)
{
    const int id = a.sid[s];
    return id >= 0 ? (unsigned short)a.atype[id] : (unsigned short)0;
}

// Synchronous staging of the folded tile + halo with species.  WITH_FP: plane
// B's zw hold F' (force pass), else |u|^2 (density pass).  Returns max |u|
// over the occupied staged sites, as stage_tile_p.
template <int TX, int TY, int TZ, bool WITH_FP>
__device__ __forceinline__ float stage_tile_pa(const GatherArgs<float> &a, const TileLoc &L, float4 *sA,
                                               unsigned short *sT, float *sred)
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
        const float fa = WITH_FP ? a.fp[sa] : xa * xa + ya * ya + za * za;
        const float fb = WITH_FP ? a.fp[sb] : xb * xb + yb * yb + zb * zb;
        umax2 = fmaxf(umax2, fmaxf(occ_u2(xa, ya, za), occ_u2(xb, yb, zb)));
        sA[p * G::PLANE + r] = make_float4(xa, xb, ya, yb);
        sB[p * G::PLANE + r] = make_float4(za, zb, fa, fb);
        sT[p * G::PLANE + r] = (unsigned short)(site_species(a, sa) | (site_species(a, sb) << 8));
    }
    return sqrtf(block_max<G::NT>(umax2, sred)) * 1.000001f;
}

__device__ __forceinline__ float4 tex4(unsigned long long tex, int i)
{
    return tex1Dfetch<float4>((cudaTextureObject_t)tex, i);
}

__device__ __forceinline__ float quad(const float4 c, float t) { return fmaf(fmaf(c.x, t, c.y), t, c.z); }

// density spline coefficients of neighbour species j at window segment i:
// the shared-memory window for the dominant species, the texture path else
__device__ __forceinline__ float4 dens_coef(const float4 *__restrict__ tab, int m, unsigned long long texv, int n,
                                            int seg_lo, int j, int i)
{
    float4 c;
    if (j == m) c = tab[i];
    else c = tex4(texv, j * n + seg_lo + i);
    return c;
}

template <int SH>
__device__ __forceinline__ void density_shells_pa(const ShellInfo &shc, int seg_lo, const float4 *__restrict__ po,
                                                  const float4 *__restrict__ sA, const float4 *__restrict__ sB,
                                                  const unsigned short *__restrict__ sT, int slot, const PairSites &ui,
                                                  float2 unorm, float rc_lat, float2 lim2, float2 S2, unsigned nwin,
                                                  const float4 *__restrict__ tab, int m, unsigned long long texv, int n,
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
                const unsigned ty = sT[slot + D];
                float2 t, rs;
                int ia, ib;
                arg_p(sh, g.q, S2, nwin, t, rs, ia, ib);
                const float4 ca = dens_coef(tab, m, texv, n, seg_lo, (int)(ty & 0xffu), ia);
                const float4 cb = dens_coef(tab, m, texv, n, seg_lo, (int)(ty >> 8), ib);
                part = p_add(part, make_float2(cubic(ca, t.x), cubic(cb, t.y)));
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
                    const unsigned ty = sT[slot + D];
                    float2 t, rs;
                    int ia, ib;
                    arg_p(sh, g.q, S2, nwin, t, rs, ia, ib);
                    const float4 ca = dens_coef(tab, m, texv, n, seg_lo, (int)(ty & 0xffu), ia);
                    const float4 cb = dens_coef(tab, m, texv, n, seg_lo, (int)(ty >> 8), ib);
                    part = p_add(part, make_float2(cubic(ca, t.x), cubic(cb, t.y)));
                    const int bi = k - kSparseK0;
                    if (bi < 64) {
                        const unsigned long long bit = 1ull << bi;
                        if (ia < (int)nwin) ma |= bit;
                        if (ib < (int)nwin) mb |= bit;
                    }
                }
            }
        }
        kahan_nz(ra, part.x);
        kahan_nz(rb, part.y);
        density_shells_pa<SH + 1>(shc, seg_lo, po, sA, sB, sT, slot, ui, unorm, rc_lat, lim2, S2, nwin, tab, m, texv, n,
                                  ra, rb, ma, mb);
    }
}

// species of the thread's two sites and their table offsets
struct PSpecies {
    int ta, tb;    // species of sites a, b
    int oa, ob;    // ta * n, tb * n
};

struct AlloyTex {
    unsigned long long fd, pd;  // density derivative per species, pair derivative per pair
    int n, nsp;
};

// one candidate of the alloy force pass for both sites
template <bool ENERGY>
__device__ __forceinline__ void force_pair_pa(const PShell &sh, const PGeom &g, const float4 B, unsigned ty,
                                              const PairSites &ui, const PSpecies &si, float2 S2, unsigned nwin,
                                              const AlloyTex &tx, const Vec4<float> *__restrict__ tpv, float2 &px,
                                              float2 &py, float2 &pz, double &ea, double &eb)
{
    float2 t, rs;
    int ia, ib;
    arg_p(sh, g.q, S2, nwin, t, rs, ia, ib);
    const int ja = (int)(ty & 0xffu), jb = (int)(ty >> 8);
    const int pa = alloy_pair(si.ta, ja, tx.nsp) * tx.n + ia, pb = alloy_pair(si.tb, jb, tx.nsp) * tx.n + ib;
    // rho' of the neighbour's species: the site's own fetch when the two
    // species agree (the pass is bound by texture fetches)
    const float4 dia = tex4(tx.fd, si.oa + ia), dib = tex4(tx.fd, si.ob + ib);
    const float4 dja = ja == si.ta ? dia : tex4(tx.fd, ja * tx.n + ia);
    const float4 djb = jb == si.tb ? dib : tex4(tx.fd, jb * tx.n + ib);
    const float4 dpa = tex4(tx.pd, pa), dpb = tex4(tx.pd, pb);
    const float2 dfj = make_float2(quad(dja, t.x), quad(djb, t.y));
    const float2 dfi = make_float2(quad(dia, t.x), quad(dib, t.y));
    const float2 dph = make_float2(quad(dpa, t.x), quad(dpb, t.y));
    // Eq. eam_force_ij: F'_i rho'_{t_j} + F'_j rho'_{t_i} + phi'_{t_i t_j}, over r
    const float2 sc = p_mul(p_fma(ui.fp, dfj, p_fma(make_float2(B.z, B.w), dfi, dph)), rs);
    px = p_fma(sc, p_fma(p_dup(0.5f), g.nx2, g.dx), px);
    py = p_fma(sc, p_fma(p_dup(0.5f), g.ny2, g.dy), py);
    pz = p_fma(sc, p_fma(p_dup(0.5f), g.nz2, g.dz), pz);
    if (ENERGY) {
        const int ua = (int)nwin;
        if (ia < ua) ea += 0.5 * (double)cubic(*reinterpret_cast<const float4 *>(&tpv[pa]), t.x);
        if (ib < ua) eb += 0.5 * (double)cubic(*reinterpret_cast<const float4 *>(&tpv[pb]), t.y);
    }
}

template <int SH, bool ENERGY>
__device__ __forceinline__ void force_shells_pa(const ShellInfo &shc, const float4 *__restrict__ po,
                                                const float4 *__restrict__ sA, const float4 *__restrict__ sB,
                                                const unsigned short *__restrict__ sT, int slot, const PairSites &ui,
                                                const PSpecies &si, float2 lim2, float2 S2, unsigned nwin,
                                                const AlloyTex &tx, const Vec4<float> *__restrict__ tpv, bool use_mask,
                                                unsigned long long msk, Acc<float> (&fa)[3], Acc<float> (&fb)[3],
                                                double &ea, double &eb)
{
    if constexpr (SH < kLVec.nshell) {
        constexpr int KB = kLVec.shell_begin[SH], KE = kLVec.shell_begin[SH + 1];
        constexpr int N2 = kLVec.shell_n2[SH];
        constexpr bool dense = SH < kSparseShell;
        const bool na = (float)N2 <= lim2.x, nb = (float)N2 <= lim2.y;
        if (SH >= shc.nshell || !(na || nb)) return;
        const PShell sh = pshell<SH>(shc, 0);
        float2 px = make_float2(0.f, 0.f), py = px, pz = px;
        if (dense || !use_mask) {
#pragma unroll 2
            for (int k = KB; k < KE; ++k) {
                const float4 o0 = po[2 * k], o1 = po[2 * k + 1];
                const int D = __float_as_int(o1.z);
                const float4 B = sB[slot + D];
                const PGeom g = pair_geom(o0, o1, sA[slot + D], B, ui);
                if (dense || g.q.x < sh.thr || g.q.y < sh.thr)
                    force_pair_pa<ENERGY>(sh, g, B, sT[slot + D], ui, si, S2, nwin, tx, tpv, px, py, pz, ea, eb);
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
                force_pair_pa<ENERGY>(sh, g, B, sT[slot + D], ui, si, S2, nwin, tx, tpv, px, py, pz, ea, eb);
            }
        }
        kahan3_nz(fa, px.x, py.x, pz.x);
        kahan3_nz(fb, px.y, py.y, pz.y);
        force_shells_pa<SH + 1, ENERGY>(shc, po, sA, sB, sT, slot, ui, si, lim2, S2, nwin, tx, tpv, use_mask, msk, fa, fb,
                                        ea, eb);
    }
}

// run-away neighbours of one site (species in the staged record's w)
__device__ __forceinline__ void ra_density_site_a(const GatherArgs<float> &a, const TileLoc &L, int cnt,
                                                  const int4 *rh, const Vec4<float> *ru, const Vec4<float> &ui, int sx,
                                                  int sy, int sz, Acc<float> &rho, unsigned &st)
{
    for (int j = 0; j < cnt; ++j) {
        const int4 h = rh[j];
        const RaPair<float> P = ra_pair<float>(a, L.rd, h, ru[j], ui, sx, sy, sz);
        if (P.in) {
            if (P.floor_hit) st |= kStRfloor;
            rho.add(cubic(tex4(a.tex_afv, h.w * a.nknot + P.seg), P.t));
        }
    }
}

template <bool ENERGY>
__device__ __forceinline__ void ra_force_site_a(const GatherArgs<float> &a, const TileLoc &L, int cnt, const int4 *rh,
                                                const Vec4<float> *ru, const Vec4<float> &ui, int ti, int sx, int sy,
                                                int sz, Acc<float> (&f)[3], double &e, unsigned &st)
{
    const int n = a.nknot;
    for (int j = 0; j < cnt; ++j) {
        const int4 h = rh[j];
        const Vec4<float> uj = ru[j];
        const RaPair<float> P = ra_pair<float>(a, L.rd, h, uj, ui, sx, sy, sz);
        if (P.in) {
            const int pr = alloy_pair(ti, h.w, a.nsp) * n + P.seg;
            const float dfj = quad(tex4(a.tex_afd, h.w * n + P.seg), P.t);
            const float dfi = quad(tex4(a.tex_afd, ti * n + P.seg), P.t);
            const float dph = quad(tex4(a.tex_apd, pr), P.t);
            const float coef = ui.w * dfj + uj.w * dfi + dph;
            const float sc_ = P.floor_hit ? 0.f : coef * P.rinv;
            if (P.floor_hit) st |= kStRfloor;
            f[0].add(sc_ * P.rx);
            f[1].add(sc_ * P.ry);
            f[2].add(sc_ * P.rz);
            if (ENERGY) e += 0.5 * (double)cubic(*reinterpret_cast<const float4 *>(&a.al_tpv[pr]), P.t);
        }
    }
}

// ---------------------------------------------------------------------------
// density pass: rho_i, F'(rho_i) with species
// ---------------------------------------------------------------------------

template <int TX, int TY, int TZ, bool ENERGY>
__global__ void __launch_bounds__(TX *TY *TZ, 1) k_density_pa(const __grid_constant__ GatherArgs<float> a)
{
    using G = PTile<TX, TY, TZ>;
    extern __shared__ __align__(32) unsigned char smem[];
    const int nwin = a.nseg - a.seg_lo;
    const int n = a.nknot, m = a.amaj;
    // the dominant species' density window plus the zero segment
    float4 *tab = reinterpret_cast<float4 *>(smem);
    for (int k = threadIdx.x; k <= nwin; k += G::NT) {
        const Vec4<float> c = k < nwin ? a.al_tfv[(size_t)m * n + a.seg_lo + k] : Vec4<float>{0.f, 0.f, 0.f, 0.f};
        tab[k] = make_float4(c.x, c.y, c.z, c.w);
    }
    const size_t wb = alloy_window_bytes(false, nwin);
    const PackedSmem sm = carve_p<TX, TY, TZ>(smem, wb, 1);
    unsigned short *sT =
        reinterpret_cast<unsigned short *>(smem + ((packed_smem_bytes(wb, TX, TY, TZ, 1) + 255) & ~(size_t)255));
    fill_rep_cache<float>(a, sm.rep);
    __syncthreads();

    const PThread<TX, TY, TZ> th;
    const float4 *po = &a.offp[th.p][0][0];
    const float2 S2 = p_dup(a.S);
    unsigned st = 0;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        double dt_rep;
        int nra;
        const TileLoc L = locate_cached(a, sm.rep, tile, TX, TY, TZ, dt_rep, nra);
        float4 *cA = sm.tA;
        const float4 *cB = cA + 2 * G::PLANE;
        __syncthreads();  // every read of the previous tile is done
        const float U = stage_tile_pa<TX, TY, TZ, false>(a, L, cA, sT, sm.red);
        const bool has_ra = a.tile_flag[tile] != 0 && nra > 0;
        const bool in_xy = (L.c0x + th.lx < L.rd.nx) && (L.c0y + th.ly < L.rd.ny);
        const bool in_a = in_xy && (L.c0z + th.lz < L.rd.nz);
        const bool in_b = in_xy && (L.c0z + th.lz + G::HZ < L.rd.nz);
        const float4 A = cA[th.slot], B = cB[th.slot];
        const unsigned tyo = sT[th.slot];
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
            density_shells_pa<0>(a.sh, a.seg_lo, po, cA, cB, sT, th.slot, ui, un, a.rc_lat, lim2, S2, (unsigned)nwin,
                                 tab, m, a.tex_afv, n, ra, rb, ma, mb);
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
                if (live_a) ra_density_site_a(a, L, cnt, sm.rh, sm.ru, ua, sx, sy, sza, ra, st);
                if (live_b) ra_density_site_a(a, L, cnt, sm.rh, sm.ru, ub, sx, sy, szb, rb, st);
                if (pos >= nra) break;
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const bool in = h ? in_b : in_a;
            if (!in) continue;
            const long long sid = site_of(L, th.lx, th.ly, th.lz + h * G::HZ, th.p);
            if (!(h ? live_b : live_a)) {
                a.fp_out[sid] = 0.f;
                continue;
            }
            if (a.mask_ok) a.bmask[sid] = h ? mb : ma;
            const float rh = (h ? rb : ra).value();
            const int ti = (int)(h ? (tyo >> 8) : (tyo & 0xffu));
            float dF;
            const float Fv = embed<float>(a.al_tFv + (size_t)ti * n, a.nseg, a.Srho, a.rho_max, rh, dF, st);
            a.fp_out[sid] = dF;
            if (ENERGY) {
                a.rho_out[sid] = rh;
                a.e_out[sid] = (double)Fv;
            }
        }
    }
    if (st) atomicOr(&a.sc[0].status, st);
}

// ---------------------------------------------------------------------------
// force pass + closing half kick with species
// ---------------------------------------------------------------------------

// Two CTAs per SM for tiles of up to 512 threads: the pass waits on texture
// latency, and more resident warps hide more of it.
template <int TX, int TY, int TZ>
constexpr int kForcePaBlocks = TX * TY * TZ <= 512 ? 2 : 1;

template <int TX, int TY, int TZ, bool ENERGY>
__global__ void __launch_bounds__(TX *TY *TZ, kForcePaBlocks<TX, TY, TZ>) k_force_pa(const __grid_constant__ GatherArgs<float> a)
{
    using G = PTile<TX, TY, TZ>;
    extern __shared__ __align__(32) unsigned char smem[];
    const PackedSmem sm = carve_p<TX, TY, TZ>(smem, 0, 1);
    unsigned short *sT =
        reinterpret_cast<unsigned short *>(smem + ((packed_smem_bytes(0, TX, TY, TZ, 1) + 255) & ~(size_t)255));
    fill_rep_cache<float>(a, sm.rep);
    __syncthreads();

    const PThread<TX, TY, TZ> th;
    const float4 *po = &a.offp[th.p][0][0];
    const float2 S2 = p_dup(a.S);
    const float conv = (float)a.acc_conv;
    const unsigned nwin = (unsigned)a.nseg;
    const AlloyTex tx{a.tex_afd, a.tex_apd, a.nknot, a.nsp};
    unsigned st = 0;
    int cur_rep = -1;
    unsigned long long vmax2 = 0;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        double dt_rep;
        int nra;
        const TileLoc L = locate_cached(a, sm.rep, tile, TX, TY, TZ, dt_rep, nra);
        if (a.kick && L.rep != cur_rep) {
            if (cur_rep >= 0) flush_vmax<G::NT>(__longlong_as_double((long long)vmax2), sm.red, a.sc + cur_rep);
            cur_rep = L.rep;
            vmax2 = 0;
        }
        float4 *cA = sm.tA;
        const float4 *cB = cA + 2 * G::PLANE;
        __syncthreads();
        const float U = stage_tile_pa<TX, TY, TZ, true>(a, L, cA, sT, sm.red);
        const double hdt = 0.5 * dt_rep;
        const bool has_ra = a.tile_flag[tile] != 0 && nra > 0;
        const bool in_xy = (L.c0x + th.lx < L.rd.nx) && (L.c0y + th.ly < L.rd.ny);
        const bool in_a = in_xy && (L.c0z + th.lz < L.rd.nz);
        const bool in_b = in_xy && (L.c0z + th.lz + G::HZ < L.rd.nz);
        const float4 A = cA[th.slot], B = cB[th.slot];
        const unsigned tyo = sT[th.slot];
        PairSites ui;
        ui.ux = make_float2(A.x, A.y);
        ui.uy = make_float2(A.z, A.w);
        ui.uz = make_float2(B.x, B.y);
        ui.fp = make_float2(B.z, B.w);
        PSpecies si;
        si.ta = (int)(tyo & 0xffu);
        si.tb = (int)(tyo >> 8);
        si.oa = si.ta * a.nknot;
        si.ob = si.tb * a.nknot;
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
            force_shells_pa<0, ENERGY>(a.sh, po, cA, cB, sT, th.slot, ui, si, lim2, S2, nwin, tx, a.al_tpv,
                                       a.mask_ok != 0, msk, fa, fb, ea, eb);
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
                if (live_a) ra_force_site_a<ENERGY>(a, L, cnt, sm.rh, sm.ru, ua, si.ta, sx, sy, sza, fa, ea, st);
                if (live_b) ra_force_site_a<ENERGY>(a, L, cnt, sm.rh, sm.ru, ub, si.tb, sx, sy, szb, fb, eb, st);
                if (pos >= nra) break;
            }
        }
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
    if (a.kick && cur_rep >= 0) flush_vmax<G::NT>(__longlong_as_double((long long)vmax2), sm.red, a.sc + cur_rep);
    if (st) atomicOr(&a.sc[0].status, st);
}

}  // namespace misa
