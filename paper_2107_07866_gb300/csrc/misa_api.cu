// misa_api.cu -- host runtime and C ABI (include/misa.h) of the GB300 EAM
// lattice-list MD library.  Owns device memory, builds the neighbour offset
// index for the chosen tile shape (Sec. 3), the replica table of a batch, and
// launches the step kernels on the handle's stream (directly, or as one
// captured CUDA graph per step).  No host fallback: every step of the path
// runs in the kernels of misa_kernels.cuh / misa_md.cuh.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "misa.h"
#include "misa_adjoint.cuh"
#include "misa_newton3.cuh"
#include "misa_packed.cuh"
#include "misa_alloy.cuh"
#include "misa_alloy_packed.cuh"
#include "misa_tiles.cuh"

using namespace misa;

namespace {

// |n| S split into integer and fraction for every |n|^2 (see SplitN2)
void fill_split(SplitN2 *sp, double S)
{
    for (int n2 = 0; n2 <= kMaxN2; ++n2) {
        const double x0 = std::sqrt((double)n2) * S, xi = std::floor(x0);
        sp[n2] = SplitN2{(float)std::sqrt((double)n2), (float)(x0 - xi), (int)xi, 0};
    }
}

// Self-test of the integer-pipe conversions against the hardware ones on
// generated bit patterns: [0] double -> float, [1] float -> double.  A
// subnormal hardware result is matched by a zero of the same sign.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void k_selftest_conv(unsigned long long n, unsigned long long *bad)
{
    unsigned long long b0 = 0, b1 = 0;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long h = mix64(i);
        unsigned long long bits = h;
        const unsigned long long keep = 0x800fffffffffffffull;
        switch (i % 4) {
        case 0:  // binary32 normal range
            bits = (h & keep) | ((897ull + (h >> 52) % 254ull) << 52);
            break;
        case 1:  // exact halfway between two binary32 values
            bits = (((h & keep) | ((897ull + (h >> 52) % 254ull) << 52)) & ~0x1fffffffull) | 0x10000000ull;
            break;
        case 2:  // any exponent
            break;
        default:  // around the binary32 underflow and overflow thresholds
            bits = (h & keep) | ((((h >> 52) & 1ull) ? 860ull + (h >> 53) % 40ull : 1140ull + (h >> 53) % 20ull) << 52);
        }
        const double d = __longlong_as_double((long long)bits);
        const float want = __double2float_rn(d), got = d2f_bits(d);
        const unsigned wb = __float_as_uint(want), gb = __float_as_uint(got);
        const bool wsub = (wb & 0x7f800000u) == 0u && (wb & 0x7fffffu) != 0u;
        if (!(wb == gb || (want != want && got != got) || (wsub && gb == (wb & 0x80000000u)))) ++b0;
        const float f = __uint_as_float((unsigned)(h >> 32) ^ (unsigned)h);
        const double wd = (double)f, gd = f2d_bits(f);
        const unsigned long long wdb = (unsigned long long)__double_as_longlong(wd);
        const unsigned long long gdb = (unsigned long long)__double_as_longlong(gd);
        const unsigned fb = __float_as_uint(f);
        const bool fsub = (fb & 0x7f800000u) == 0u && (fb & 0x7fffffu) != 0u;
        if (!(wdb == gdb || (wd != wd && gd != gd) || (fsub && gdb == ((unsigned long long)(fb >> 31) << 63)))) ++b1;
    }
    if (b0) atomicAdd(bad, b0);
    if (b1) atomicAdd(bad + 1, b1);
}

// nearest_site_fast against nearest_site (site and displacement bits) on
// positions in half-lattice units: thermal, near floor and decision ties,
// exact ties, uniform, and far outside the box.
__global__ void k_selftest_site(unsigned long long n, unsigned long long *bad)
{
    unsigned long long b = 0;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long h = mix64(i), g = mix64(i ^ 0x9e3779b97f4a7c15ull);
        const int nb = 2 + (int)(h % 600ull);
        const double L = 2.0 * nb;
        double P[3];
        for (int d = 0; d < 3; ++d) {
            const unsigned long long q = mix64(h + 31ull * d + 7ull);
            const double k = (double)(q % (unsigned long long)(2 * nb));
            const double v = (double)(q >> 11) * 0x1p-53;  // [0, 1)
            switch ((i + (unsigned long long)d * (g & 1ull)) % 6ull) {
            case 0:  // thermal
                P[d] = k + (v - 0.5) * 0.4;
                break;
            case 1:  // a few ulps around an integer (floor ties)
                P[d] = k + (double)((long long)(q >> 60) - 8) * 0x1p-52 * (k + 1.0);
                break;
            case 2:  // around a half-integer (distance ties between the sublattices)
                P[d] = k + 0.5 + (double)((long long)(q >> 60) - 8) * 0x1p-40;
                break;
            case 3:  // exact half-integer
                P[d] = k + 0.5;
                break;
            case 4:  // uniform in the box
                P[d] = v * L;
                break;
            default:  // FP32-scale offsets from an integer
                P[d] = k + (double)((long long)(q >> 58) - 32) * 0x1p-24 * (k + 2.0) * 0.05;
            }
        }
        double ax, ay, az, bx, by, bz;
        const long long sa = nearest_site(P[0], P[1], P[2], nb, nb, nb, ax, ay, az);
        const long long sb = nearest_site_fast(P[0], P[1], P[2], nb, nb, nb, bx, by, bz);
        if (sa != sb || __double_as_longlong(ax) != __double_as_longlong(bx) ||
            __double_as_longlong(ay) != __double_as_longlong(by) || __double_as_longlong(az) != __double_as_longlong(bz))
            ++b;
    }
    if (b) atomicAdd(bad, b);
}

constexpr double kAccUnit = 9.6485332123310018e-3;  // 1 eV/(A amu) in A/fs^2 (CODATA 2018)
constexpr double kRfloor = 1e-4;                      // A

std::string g_create_error;

}  // namespace

struct misa_sim {
    misa_params p{};
    std::vector<double> fk, pk, Fk;
    cudaStream_t st = nullptr;   // caller's stream
    cudaStream_t gst = nullptr;  // internal stream the step graph is captured on
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int nrep = 1;
    std::vector<int> dims;       // 3 per replica
    std::vector<RepDesc> reps;   // host copy of the replica table
    long long ns = 0;            // sites (= atoms) of all replicas
    int prec = MISA_FP32_FORCE;
    int cap = 0;                 // run-away capacity per replica
    int tile = 0;
    int nsm = 0;
    std::string err;
    std::vector<std::pair<void *, size_t>> allocs;
    // device buffers
    RepDesc *reps_d = nullptr;   // replica table with the density pass's tile counts
    int *tile_rep = nullptr;
    int *sid = nullptr, *claim = nullptr, *tile_flag = nullptr;
    // the force pass's own tile shape: replica table, tile -> replica map, run-away tile flags
    int tile_f = 0, ntiles_f = 0;
    RepDesc *reps_fd = nullptr;
    int *tile_rep_f = nullptr, *tile_flag_f = nullptr;
    // per-tile run-away index of each map (0 density, 1 force): counts,
    // segment offsets, fill cursors, tiles with run-aways, [cursor, count],
    // and the segments of sorted list indices (rt_cap entries)
    int *rt_cnt[2] = {}, *rt_off[2] = {}, *rt_fill[2] = {}, *rt_nz[2] = {}, *rt_aux[2] = {}, *rt_list[2] = {};
    long long rt_cap = 0;
    double *u[3] = {}, *v[3] = {};
    void *s[3] = {};  // precision-T shadow of u (FP32 path) or alias of u
    void *a[3] = {};
    void *fp = nullptr, *rho = nullptr;
    double *esite = nullptr;
    unsigned long long *bmask = nullptr;  // FP32: sparse-shell candidates inside rc, per site
    unsigned long long tex_f = 0, tex_d0 = 0, tex_d1 = 0;  // FP32: texture objects over the tables
    int *ra_home = nullptr, *ra_id = nullptr;
    double *ra_u[3] = {}, *ra_v[3] = {};
    void *ra_s[3] = {}, *ra_a[3] = {};
    void *ra_fp = nullptr, *ra_rho = nullptr;
    double *ra_e = nullptr;
    int *t_home = nullptr, *t_id = nullptr;
    double *t_u[3] = {}, *t_v[3] = {};
    void *t_s[3] = {}, *t_a[3] = {};
    double *knots = nullptr;
    void *tab_f = nullptr, *tab_phi = nullptr, *tab_F = nullptr, *tab_d0 = nullptr, *tab_d1 = nullptr;
    DevScalars *sc = nullptr;
    double *partial = nullptr, *red_out = nullptr;
    double *out_buf = nullptr;  // 3 natoms scratch for read-out / set_state
    int *aux_int = nullptr;     // natoms scratch
    double *aux_dbl = nullptr;  // 3 natoms scratch
    // staged state (misa_stage_state): x, v copied on the handle's copy
    // stream into buffers of their own, consumed by misa_set_state_staged
    cudaStream_t cst = nullptr;
    cudaEvent_t ev_stg = nullptr;       // the staged copies are complete
    cudaEvent_t ev_stg_free = nullptr;  // the last staged state has been read
    double *stg_x = nullptr, *stg_v = nullptr;
    bool stg_pending = false, stg_has_v = false;
    // asynchronous per-atom energies (misa_get_energies_async): written into
    // e_buf on the handle's stream, copied out on an output stream of their own
    cudaStream_t ost = nullptr;
    cudaEvent_t ev_e_ready = nullptr;  // e_buf holds the energies to copy
    cudaEvent_t ev_e_done = nullptr;   // the last copy out of e_buf is complete
    double *e_buf = nullptr;
    long long ntile_cap = 0;    // tile_flag / tile_rep capacity (smallest tile shape)
    int ntiles = 0;
    size_t smem_density = 0, smem_force = 0;
    size_t smem_alloy_d = 0, smem_alloy_f = 0;  // FP32 alloy passes (density, force tile shape)
    bool dens_db = false;  // FP32 density pass double-buffers its tiles
    bool dens_n3 = false;  // FP32 density pass with Newton's third law inside tiles
    long long launches = 0;
    // phase timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    // adjoint work arrays (allocated on first use)
    void *lam[3] = {}, *ra_lam[3] = {};
    void *dl = nullptr, *ra_dl = nullptr, *cw = nullptr;
    double *adj_partial = nullptr, *adj_sum = nullptr, *adj_grad = nullptr, *adj_eref = nullptr, *adj_fref = nullptr;
    int adj_cta = 0;
    // alloys (misa_set_species): species per atom id, coefficient tables
    int nsp = 1;
    int8_t *atype = nullptr;
    double *al_knots = nullptr;
    void *al_fv = nullptr, *al_fd = nullptr, *al_Fv = nullptr, *al_pv = nullptr, *al_pd = nullptr;
    int al_cap = 0;  // species the alloy arrays were allocated for
    int amaj = 0;    // the species with the most atoms
    unsigned long long tex_afv = 0, tex_afd = 0, tex_apd = 0;  // FP32: texture objects over the alloy tables
    // captured step graph
    bool use_graph = true;
    cudaGraphExec_t graph = nullptr;
    long long graph_launches = 0;  // kernels inside one replay
    cudaGraphExec_t graph_e = nullptr;  // the same step with per-atom energies in its force passes
    long long graph_e_launches = 0;
    bool energy_valid = false;  // esite / ra_e hold the energies of the current positions
    // the per-tile run-away index matches the current run-away list and tile
    // maps (a force evaluation outside a step then skips its rebuild); a step
    // being captured into a graph always rebuilds it
    bool ra_index_valid = false;
    bool capturing = false;
    // kick/drift block map (replica, first site) and its host copy
    int2 *kd_map = nullptr;
    int kd_blocks = 0, kd_chunk = 0;
    std::vector<int2> kd_host;
};

namespace {

int fail(misa_sim *s, int code, const std::string &msg)
{
    if (s) s->err = msg;
    else g_create_error = msg;
    return code;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(s, MISA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// drops the captured step graphs (tile shapes, tables or species changed)
void drop_graphs(misa_sim *s)
{
    if (s->graph) cudaGraphExecDestroy(s->graph);
    if (s->graph_e) cudaGraphExecDestroy(s->graph_e);
    s->graph = s->graph_e = nullptr;
}

void *dalloc(misa_sim *s, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (s->p.alloc) {
        p = s->p.alloc(bytes, s->p.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        p = nullptr;
    }
    if (p) {
        s->allocs.emplace_back(p, bytes);
        cudaMemsetAsync(p, 0, bytes, s->st);
    }
    return p;
}

// records a timing event on the stream (no-op unless timing is enabled)
void mark(misa_sim *s)
{
    if (!s->timing) return;
    if (s->ev_used == s->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        s->ev_pool.push_back(e);
    }
    cudaEvent_t e = s->ev_pool[s->ev_used++];
    cudaEventRecord(e, s->st);
}

// launch geometry: 2-D grids, x = blocks per replica, y = replica
dim3 site_grid(const misa_sim *s)
{
    int gx = (s->nsm * 8 + s->nrep - 1) / s->nrep;
    return dim3(gx < 4 ? 4 : gx, s->nrep);
}
dim3 list_grid(const misa_sim *s) { return dim3(8, s->nrep); }
// blocks per replica of the two-stage sums (k_sum_stage1, k_adj_lambda): one
// 256-thread block per 256 sites of the largest replica, at most 512
int red_blocks(const misa_sim *s)
{
    long long mx = 1;
    for (const RepDesc &rd : s->reps) mx = rd.ns > mx ? rd.ns : mx;
    const long long b = (mx + 255) / 256;
    return (int)(b > 512 ? 512 : b);
}
int rep_blocks(const misa_sim *s) { return (s->nrep + 127) / 128; }

template <typename T>
MdArgs<T> md_args(misa_sim *s)
{
    MdArgs<T> m{};
    m.reps = s->reps_d;
    m.nrep = s->nrep;
    m.kd_map = s->kd_map;
    m.kd_chunk = s->kd_chunk;
    m.sid = s->sid;
    m.ux = s->u[0]; m.uy = s->u[1]; m.uz = s->u[2];
    m.sx = (T *)s->s[0]; m.sy = (T *)s->s[1]; m.sz = (T *)s->s[2];
    m.vx = s->v[0]; m.vy = s->v[1]; m.vz = s->v[2];
    m.ax = (T *)s->a[0]; m.ay = (T *)s->a[1]; m.az = (T *)s->a[2];
    m.fp = (T *)s->fp; m.rho = (T *)s->rho;
    m.esite = s->esite;
    m.claim = s->claim;
    m.ra_home = s->ra_home; m.ra_id = s->ra_id;
    m.ra_ux = s->ra_u[0]; m.ra_uy = s->ra_u[1]; m.ra_uz = s->ra_u[2];
    m.ra_sx = (T *)s->ra_s[0]; m.ra_sy = (T *)s->ra_s[1]; m.ra_sz = (T *)s->ra_s[2];
    m.ra_vx = s->ra_v[0]; m.ra_vy = s->ra_v[1]; m.ra_vz = s->ra_v[2];
    m.ra_ax = (T *)s->ra_a[0]; m.ra_ay = (T *)s->ra_a[1]; m.ra_az = (T *)s->ra_a[2];
    m.ra_fp = (T *)s->ra_fp; m.ra_rho = (T *)s->ra_rho; m.ra_e = s->ra_e;
    m.t_home = s->t_home; m.t_id = s->t_id;
    for (int d = 0; d < 3; ++d) {
        m.t_u[d] = s->t_u[d];
        m.t_v[d] = s->t_v[d];
        m.t_s[d] = (T *)s->t_s[d];
        m.t_a[d] = (T *)s->t_a[d];
    }
    m.tile_flag = s->tile_flag;
    const TileShape &ts = kTiles[s->tile];
    m.tx = ts.tx; m.ty = ts.ty; m.tz = ts.tz;
    m.sc = s->sc;
    m.half = 0.5 * s->p.a0;
    m.inv_half = 2.0 / s->p.a0;
    double sk = s->p.skin / m.half;
    m.skin2 = sk * sk;
    m.dt_max = s->p.dt_max;
    m.dx_max = s->p.dx_max;
    m.reassign_period = s->p.reassign_period > 0 ? s->p.reassign_period : 1;
    m.acc_conv = kAccUnit / s->p.mass;
    m.mass = s->p.mass;
    return m;
}

// First spline segment an array-array pair can reach: both atoms lie within
// the skin of their sites, so r >= d_nn - 2 skin (d_nn = sqrt(3)/2 a0); two
// segments of guard for rounding.  The FP32 gathers keep only the table
// segments from here on in shared memory.
int seg_lo_of(const misa_sim *s)
{
    const int n = s->p.n_knots;
    const double hr = s->p.rc / (n - 1);
    const double rlo = 0.5 * std::sqrt(3.0) * s->p.a0 - 2.0 * s->p.skin;
    int k = (int)std::floor(rlo / hr) - 2;
    if (k < 0) k = 0;
    if (k > n - 2) k = n - 2;
    return k;
}

template <typename T>
void fill_gather(misa_sim *s, GatherArgs<T> &g, bool force_pass = false)
{
    std::memset(&g, 0, sizeof(g));
    const TileShape &ts = kTiles[force_pass ? s->tile_f : s->tile];
    g.reps = force_pass ? s->reps_fd : s->reps_d;
    g.tile_rep = force_pass ? s->tile_rep_f : s->tile_rep;
    g.ntiles = force_pass ? s->ntiles_f : s->ntiles;
    g.nrep = s->nrep;
    g.ux = (const T *)s->s[0]; g.uy = (const T *)s->s[1]; g.uz = (const T *)s->s[2];
    g.fp = (const T *)s->fp;
    g.fp_out = (T *)s->fp;
    g.rho_out = (T *)s->rho;
    g.e_out = s->esite;
    g.ax = (T *)s->a[0]; g.ay = (T *)s->a[1]; g.az = (T *)s->a[2];
    g.vx = s->v[0]; g.vy = s->v[1]; g.vz = s->v[2];
    g.tab_f = (const Vec4<T> *)s->tab_f;
    g.tab_phi = (const Vec4<T> *)s->tab_phi;
    g.tab_F = (const Vec4<T> *)s->tab_F;
    g.tab_d0 = (const Vec4<T> *)s->tab_d0;
    g.tab_d1 = (const Vec2<T> *)s->tab_d1;
    const int n = s->p.n_knots;
    g.nseg = n - 1;
    g.seg_lo = seg_lo_of(s);
    const double half = 0.5 * s->p.a0;
    const double hr = s->p.rc / (n - 1);
    const double hrho = s->p.rho_max / (n - 1);
    const double S = half / hr;
    g.S = (T)S;
    g.Srho = (T)(1.0 / hrho);
    g.rho_max = (T)s->p.rho_max;
    const double rcl = s->p.rc / half;
    g.rc2 = (T)(rcl * rcl);
    g.rc_lat = (T)rcl;
    g.rfloor2 = (T)((kRfloor / half) * (kRfloor / half));
    g.ra_home = s->ra_home;
    g.ra_ux = (const T *)s->ra_s[0]; g.ra_uy = (const T *)s->ra_s[1]; g.ra_uz = (const T *)s->ra_s[2];
    g.ra_fp = (const T *)s->ra_fp;
    g.tile_flag = force_pass ? s->tile_flag_f : s->tile_flag;
    g.ra_toff = s->rt_off[force_pass ? 1 : 0];
    g.ra_tcnt = s->rt_cnt[force_pass ? 1 : 0];
    g.ra_tlist = s->rt_list[force_pass ? 1 : 0];
    g.sc = s->sc;
    g.acc_conv = kAccUnit / s->p.mass;
    g.kick = 1;
    // neighbour offset index for this tile shape (Sec. 3): per parity, the
    // shared-memory slot displacement of every lattice vector (FP32: in the
    // tile folded in z, two sites per slot)
    const int SX = ts.tx + 4, SY = ts.ty + 4, SZ = sizeof(T) == 4 ? ts.tz / 2 + 4 : ts.tz + 4;
    const int PLANE = SX * SY * SZ;
    for (int par = 0; par < 2; ++par)
        for (int k = 0; k < kNVec; ++k) {
            const LVec &o = kLVec.v[k];
            int pp = par ^ (o.x & 1);
            int D = (pp - par) * PLANE + (cell_shift(par, o.z) * SY + cell_shift(par, o.y)) * SX + cell_shift(par, o.x);
            float fD;
            std::memcpy(&fD, &D, sizeof(int));
            g.off[par][k] = make_float4(fD, 2.0f * o.x, 2.0f * o.y, 2.0f * o.z);
            g.offp[par][k][0] = make_float4(2.0f * o.x, 2.0f * o.x, 2.0f * o.y, 2.0f * o.y);
            g.offp[par][k][1] = make_float4(2.0f * o.z, 2.0f * o.z, fD, 0.f);
        }
    const double roff = (s->p.rc + 2.0 * s->p.skin) / half;
    ShellInfo &sh = g.sh;
    sh.nshell = 0;
    for (int q = 0; q < kLVec.nshell; ++q) {
        if (kLVec.shell_n2[q] > roff * roff) break;
        int n2 = kLVec.shell_n2[q];
        sh.thr[q] = (float)(rcl * rcl - n2);
        sh.thr_d[q] = rcl * rcl - n2;
        double nr = std::sqrt((double)n2);
        sh.nrm[q] = (float)nr;
        double x0 = nr * S;
        double xi = std::floor(x0);
        sh.xoff[q] = (int)xi - 0x4B400000;
        sh.xfrac[q] = (float)(x0 - xi);
        sh.nshell = q + 1;
    }
    g.bmask = s->bmask;
    g.tex_f = s->tex_f;
    g.tex_d0 = s->tex_d0;
    g.tex_d1 = s->tex_d1;
    g.mask_ok = s->bmask && kLVec.shell_begin[sh.nshell] - kSparseK0 <= 64 ? 1 : 0;
    g.sid = s->sid;
    if (s->nsp > 1) {
        g.atype = s->atype;
        g.ra_id = s->ra_id;
        g.nsp = s->nsp;
        g.nknot = n;
        g.tex_afv = s->tex_afv;
        g.tex_afd = s->tex_afd;
        g.tex_apd = s->tex_apd;
        g.al_tFv = (const Vec4<T> *)s->al_Fv;
        g.al_tpv = (const Vec4<T> *)s->al_pv;
        g.al_tfv = (const Vec4<T> *)s->al_fv;
        g.amaj = s->amaj;
    }
}

// FP32: the table window plus one zero segment, the folded tile (two
// buffers for the density pass when they fit); FP64: tables in global memory.
template <typename T>
size_t smem_density_bytes(misa_sim *s, size_t optin)
{
    const TileShape &ts = kTiles[s->tile];
    const size_t nwin = (size_t)(s->p.n_knots - 1 - seg_lo_of(s));
    if constexpr (sizeof(T) == 4) {
        const size_t tb = sizeof(float4) * (nwin + 1);
        if (s->dens_n3) {  // plus the exchange buffer of the Newton-3 pass
            const size_t two = n3_smem_bytes(tb, ts.tx, ts.ty, ts.tz, 2);
            s->dens_db = two <= optin;
            return s->dens_db ? two : n3_smem_bytes(tb, ts.tx, ts.ty, ts.tz, 1);
        }
        const size_t two = packed_smem_bytes(tb, ts.tx, ts.ty, ts.tz, 2);
        s->dens_db = two <= optin;
        return s->dens_db ? two : packed_smem_bytes(tb, ts.tx, ts.ty, ts.tz, 1);
    } else {
        s->dens_db = false;
        return gather_smem_bytes<T>(0, ts.tx, ts.ty, ts.tz, tile_buffers<T>());
    }
}

template <typename T>
size_t smem_force_bytes(misa_sim *s)
{
    const TileShape &ts = kTiles[s->tile_f];
    const size_t nwin = (size_t)(s->p.n_knots - 1 - seg_lo_of(s));
    if constexpr (sizeof(T) == 4)
        return packed_smem_bytes(sizeof(float4) * (nwin + 1), ts.tx, ts.ty, ts.tz, 1);
    else
        return gather_smem_bytes<T>(0, ts.tx, ts.ty, ts.tz, 1);
}

// the handle's side of a tile launch (misa_tiles.cuh)
TileLaunch tile_launch(const misa_sim *s)
{
    TileLaunch L;
    L.st = s->st;
    L.smem_density = s->smem_density;
    L.smem_force = s->smem_force;
    L.smem_alloy_d = s->smem_alloy_d;
    L.smem_alloy_f = s->smem_alloy_f;
    L.nsm = s->nsm;
    L.nsp = s->nsp;
    L.dens_db = s->dens_db;
    L.dens_n3 = s->dens_n3;
    return L;
}

// Tile counts of every replica for one tile shape and the global tile ->
// replica map; the tile fields of reps are overwritten.
int build_tile_map(misa_sim *s, const TileShape &ts, std::vector<RepDesc> &reps, std::vector<int> &map)
{
    int base = 0;
    map.clear();
    for (int r = 0; r < s->nrep; ++r) {
        RepDesc &rd = reps[r];
        rd.ntx = (rd.nx + ts.tx - 1) / ts.tx;
        rd.nty = (rd.ny + ts.ty - 1) / ts.ty;
        rd.ntz = (rd.nz + ts.tz - 1) / ts.tz;
        rd.ntiles = rd.ntx * rd.nty * rd.ntz;
        rd.tile_base = base;
        base += rd.ntiles;
        map.insert(map.end(), rd.ntiles, r);
    }
    return base;
}

// Sets the tile shapes of the density pass (td) and the force pass (tf):
// tile counts of every replica, the global tile -> replica maps, kernel
// attributes.  Drops a captured step graph.
template <typename T>
int configure(misa_sim *s, int td, int tf)
{
    if (!tile_ok(s->prec, kTiles[td]) || !tile_ok(s->prec, kTiles[tf]))
        return fail(s, MISA_EINVAL, "tile shape not built for this precision");
    s->tile = td;
    s->tile_f = tf;
    s->ra_index_valid = false;
    std::vector<int> map, map_f;
    std::vector<RepDesc> reps_f = s->reps;
    s->ntiles = build_tile_map(s, kTiles[td], s->reps, map);
    s->ntiles_f = build_tile_map(s, kTiles[tf], reps_f, map_f);
    if ((long long)s->ntiles > s->ntile_cap || (long long)s->ntiles_f > s->ntile_cap)
        return fail(s, MISA_EINVAL, "tile map capacity");
    CK(cudaMemcpyAsync(s->reps_d, s->reps.data(), sizeof(RepDesc) * s->nrep, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->tile_rep, map.data(), sizeof(int) * map.size(), cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->reps_fd, reps_f.data(), sizeof(RepDesc) * s->nrep, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->tile_rep_f, map_f.data(), sizeof(int) * map_f.size(), cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));  // the maps are host temporaries
    int dev = 0, optin = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    s->smem_density = smem_density_bytes<T>(s, (size_t)optin);
    s->smem_force = smem_force_bytes<T>(s);
    s->smem_alloy_d = s->smem_alloy_f = 0;
    if (sizeof(T) == 4) {
        // the alloy passes' sizes; 0 marks a shape whose alloy pass does not fit
        const TileShape &a = kTiles[td], &b = kTiles[tf];
        const int nwin = s->p.n_knots - 1 - seg_lo_of(s);
        const size_t ad = alloy_smem_bytes(false, nwin, a.tx, a.ty, a.tz);
        const size_t af = alloy_smem_bytes(true, nwin, b.tx, b.ty, b.tz);
        s->smem_alloy_d = ad <= (size_t)optin ? ad : 0;
        s->smem_alloy_f = af <= (size_t)optin ? af : 0;
        if (s->nsp > 1 && (!s->smem_alloy_d || !s->smem_alloy_f))
            return fail(s, MISA_EINVAL, "tile shape and table windows exceed the shared memory of a block (alloy passes)");
    }
    if (s->smem_density > (size_t)optin || s->smem_force > (size_t)optin)
        return fail(s, MISA_EINVAL, "tile shape and table window exceed the shared memory of a block");
    CK(tile_attrs<T>(td, false, tile_launch(s)));
    CK(tile_attrs<T>(tf, true, tile_launch(s)));
    CK(cudaFuncSetAttribute(k_ra_sort<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)(sizeof(unsigned long long) * kSortMax)));
    drop_graphs(s);
    return MISA_OK;
}

// Per-tile run-away index of both passes' tile maps (sets their tile
// flags): count, allocate segments, fill, sort each segment into list order.
template <typename T>
int mark_tiles(misa_sim *s)
{
    if (s->ra_index_valid && !s->capturing) return MISA_OK;
    MdArgs<T> m = md_args<T>(s);
    RaTileMaps Ms;
    int nt = 0;
    for (int k = 0; k < 2; ++k) {
        const TileShape &ts = kTiles[k ? s->tile_f : s->tile];
        RaTileMap &M = Ms.m[k];
        M.reps = k ? s->reps_fd : s->reps_d;
        M.tx = ts.tx; M.ty = ts.ty; M.tz = ts.tz;
        M.ntiles = k ? s->ntiles_f : s->ntiles;
        M.flag = k ? s->tile_flag_f : s->tile_flag;
        M.cnt = s->rt_cnt[k]; M.off = s->rt_off[k]; M.fill = s->rt_fill[k]; M.list = s->rt_list[k];
        M.nz = s->rt_nz[k]; M.aux = s->rt_aux[k];
        M.cap = (int)s->rt_cap;
        nt = nt > M.ntiles ? nt : M.ntiles;
    }
    // the two maps' counts and cursors are contiguous (one allocation)
    CK(cudaMemsetAsync(s->rt_cnt[0], 0, sizeof(int) * (size_t)s->ntile_cap * 2, s->st));
    CK(cudaMemsetAsync(s->rt_aux[0], 0, sizeof(int) * 4, s->st));
    const dim3 lg((s->cap + 255) / 256 < 64 ? (s->cap + 255) / 256 : 64, s->nrep);
    k_ra_tcount<T><<<lg, 256, 0, s->st>>>(m, Ms);
    const int tb = (nt + 255) / 256;
    k_ra_toff<<<tb < 1024 ? tb : 1024, 256, 0, s->st>>>(Ms);
    k_ra_tfill<T><<<lg, 256, 0, s->st>>>(m, Ms);
    k_ra_tsort<<<dim3(s->nsm, 2), 32 * kRaSortWarps, 0, s->st>>>(Ms);
    s->launches += 4;
    s->ra_index_valid = !s->capturing;
    return MISA_OK;
}

template <typename T>
void launch_density(misa_sim *s, const GatherArgs<T> &g, bool energy)
{
    const int grid = s->ntiles < s->nsm ? s->ntiles : s->nsm;
    tile_density<T>(s->tile, tile_launch(s), g, grid, energy);
}

template <typename T>
void launch_force(misa_sim *s, const GatherArgs<T> &g, bool energy)
{
    const int grid = s->ntiles_f < s->nsm ? s->ntiles_f : s->nsm;
    tile_force<T>(s->tile_f, tile_launch(s), g, grid, energy);
}

template <typename T>
AlloyArgs<T> alloy_args(misa_sim *s, int kick, bool energy)
{
    AlloyArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.reps = s->reps_d;
    a.nrep = s->nrep;
    a.sid = s->sid;
    a.ux = (const T *)s->s[0]; a.uy = (const T *)s->s[1]; a.uz = (const T *)s->s[2];
    a.fp = (T *)s->fp; a.rho_out = (T *)s->rho; a.e_out = s->esite;
    a.ax = (T *)s->a[0]; a.ay = (T *)s->a[1]; a.az = (T *)s->a[2];
    a.vx = s->v[0]; a.vy = s->v[1]; a.vz = s->v[2];
    a.ra_home = s->ra_home; a.ra_id = s->ra_id;
    a.ra_ux = (const T *)s->ra_s[0]; a.ra_uy = (const T *)s->ra_s[1]; a.ra_uz = (const T *)s->ra_s[2];
    a.ra_fp = (T *)s->ra_fp; a.ra_rho = (T *)s->ra_rho; a.ra_e = s->ra_e;
    a.ra_ax = (T *)s->ra_a[0]; a.ra_ay = (T *)s->ra_a[1]; a.ra_az = (T *)s->ra_a[2];
    a.ra_vx = s->ra_v[0]; a.ra_vy = s->ra_v[1]; a.ra_vz = s->ra_v[2];
    a.sc = s->sc;
    a.atype = s->atype;
    a.nsp = s->nsp;
    const int n = s->p.n_knots;
    a.n = n;
    a.tfv = (const Vec4<T> *)s->al_fv; a.tfd = (const Vec4<T> *)s->al_fd; a.tFv = (const Vec4<T> *)s->al_Fv;
    a.tpv = (const Vec4<T> *)s->al_pv; a.tpd = (const Vec4<T> *)s->al_pd;
    const double half = 0.5 * s->p.a0, hr = s->p.rc / (n - 1), hrho = s->p.rho_max / (n - 1);
    a.S = (T)(half / hr);
    const double rcl = s->p.rc / half;
    a.rc2 = (T)(rcl * rcl);
    a.rfloor2 = (T)((kRfloor / half) * (kRfloor / half));
    a.Srho = (T)(1.0 / hrho);
    a.rho_max = (T)s->p.rho_max;
    a.acc_conv = kAccUnit / s->p.mass;
    a.kick = kick;
    a.energy = energy ? 1 : 0;
    const double roff = (s->p.rc + 2.0 * s->p.skin) / half;
    int nsh = 0;
    while (nsh < kLVec.nshell && kLVec.shell_n2[nsh] <= roff * roff) ++nsh;
    a.nvec = kLVec.shell_begin[nsh];
    a.tile_flag = s->tile_flag;
    a.ra_toff = s->rt_off[0]; a.ra_tcnt = s->rt_cnt[0]; a.ra_tlist = s->rt_list[0];
    const TileShape &ts = kTiles[s->tile];
    a.tx = ts.tx; a.ty = ts.ty; a.tz = ts.tz;
    fill_split(a.split, half / hr);
    return a;
}

// the four alloy passes (density, run-away density, force + kick, run-away
// force + kick): FP32 the packed tile gathers with species (array atoms),
// FP64 one thread per site
template <typename T>
int launch_alloy(misa_sim *s, int kick, bool energy, bool step_marks)
{
    int rc = mark_tiles<T>(s);
    if (rc) return rc;
    const AlloyArgs<T> a = alloy_args<T>(s, kick, energy);
    GatherArgs<T> gd, gf;
    if constexpr (sizeof(T) == 4) {
        fill_gather<T>(s, gd, false);
        fill_gather<T>(s, gf, true);
        gd.kick = gf.kick = kick;
    }
    if (step_marks) mark(s);
    if constexpr (sizeof(T) == 4) launch_density<T>(s, gd, energy);
    else k_alloy_density<T><<<site_grid(s), 256, 0, s->st>>>(a);
    if (step_marks) mark(s);
    k_alloy_ra_density<T><<<dim3(16, s->nrep), 256, 0, s->st>>>(a);
    if (step_marks) mark(s);
    if constexpr (sizeof(T) == 4) launch_force<T>(s, gf, energy);
    else k_alloy_force<T><<<site_grid(s), 256, 0, s->st>>>(a);
    if (step_marks) mark(s);
    k_alloy_ra_force<T><<<dim3(16, s->nrep), 256, 0, s->st>>>(a);
    if (step_marks) mark(s);
    s->launches += 6;
    CK(cudaGetLastError());
    return MISA_OK;
}

template <typename T>
int launch_forces(misa_sim *s, int kick, bool energy, bool step_marks = false)
{
    if (s->nsp > 1) return launch_alloy<T>(s, kick, energy, step_marks);
    GatherArgs<T> gd, gf;
    fill_gather<T>(s, gd, false);
    fill_gather<T>(s, gf, true);
    gd.kick = gf.kick = kick;
    int rc = mark_tiles<T>(s);
    if (rc) return rc;
    RaGatherArgs<T> ra;
    std::memset(&ra, 0, sizeof(ra));
    ra.g = gd;
    ra.g.kick = kick;
    ra.sid = s->sid;
    ra.ra_sx = (const T *)s->ra_s[0]; ra.ra_sy = (const T *)s->ra_s[1]; ra.ra_sz = (const T *)s->ra_s[2];
    ra.ra_fp = (T *)s->ra_fp; ra.ra_rho = (T *)s->ra_rho; ra.ra_e = s->ra_e;
    ra.ra_ax = (T *)s->ra_a[0]; ra.ra_ay = (T *)s->ra_a[1]; ra.ra_az = (T *)s->ra_a[2];
    ra.ra_vx = s->ra_v[0]; ra.ra_vy = s->ra_v[1]; ra.ra_vz = s->ra_v[2];
    ra.energy = energy ? 1 : 0;
    ra.tx = kTiles[s->tile].tx; ra.ty = kTiles[s->tile].ty; ra.tz = kTiles[s->tile].tz;
    // one warp per run-away (grid-stride): four CTAs of 8 warps per SM over
    // all replicas, at least 16 per replica, never more than a full list
    int rab = 4 * s->nsm / s->nrep;
    if (rab < 16) rab = 16;
    if (rab > (s->cap + 7) / 8) rab = (s->cap + 7) / 8 > 16 ? (s->cap + 7) / 8 : 16;
    if (step_marks) mark(s);  // end of the list phase
    launch_density<T>(s, gd, energy);
    if (step_marks) mark(s);
    k_ra_gather<T, 0><<<dim3(rab, s->nrep), 256, 0, s->st>>>(ra);
    if (step_marks) mark(s);
    launch_force<T>(s, gf, energy);
    if (step_marks) mark(s);
    k_ra_gather<T, 1><<<dim3(rab, s->nrep), 256, 0, s->st>>>(ra);
    if (step_marks) mark(s);
    s->launches += 6;
    CK(cudaGetLastError());
    return MISA_OK;
}

// the launches of one MD step on s->st
template <typename T>
int launch_step(misa_sim *s, bool energy = false)
{
    MdArgs<T> m = md_args<T>(s);
    s->ra_index_valid = false;  // the list phase below changes the run-away list
    mark(s);
    k_begin_step<T><<<rep_blocks(s), 128, 0, s->st>>>(m);
    k_ra_kick_drift<T><<<list_grid(s), 256, 0, s->st>>>(m);
    k_kick_drift<T><<<s->kd_blocks, 256, 0, s->st>>>(m);
    mark(s);
    k_reassign_claim<T><<<list_grid(s), 256, 0, s->st>>>(m, 0);
    k_reassign_promote<T><<<list_grid(s), 256, 0, s->st>>>(m, 0);
    k_ra_sort<T><<<s->nrep, 1024, sizeof(unsigned long long) * kSortMax, s->st>>>(m);
    s->launches += 6;
    int rc = launch_forces<T>(s, 1, energy, true);
    if (rc) return rc;
    k_end_step<T><<<rep_blocks(s), 128, 0, s->st>>>(m);
    mark(s);
    s->launches += 1;
    CK(cudaGetLastError());
    return MISA_OK;
}

// One step captured as a CUDA graph on an internal stream (a second graph
// for the step whose force passes also evaluate per-atom energies), replayed
// n times, the last one the energy step when asked; the caller's stream is
// joined by events.
template <typename T>
int capture_step(misa_sim *s, bool energy, cudaGraphExec_t *out, long long *launches)
{
    cudaStream_t user = s->st;
    s->st = s->gst;
    long long l0 = s->launches;
    CK(cudaStreamBeginCapture(s->gst, cudaStreamCaptureModeThreadLocal));
    s->capturing = true;
    int rc = launch_step<T>(s, energy);
    s->capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s->gst, &g);
    s->st = user;
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(s, MISA_ECUDA, std::string("step capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(s, MISA_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    *launches = s->launches - l0;
    s->launches = l0;
    return MISA_OK;
}

template <typename T>
int step_graph(misa_sim *s, int n, bool energy_last = false)
{
    const int plain = energy_last ? n - 1 : n;
    if (plain > 0 && !s->graph) {
        int rc = capture_step<T>(s, false, &s->graph, &s->graph_launches);
        if (rc) return rc;
    }
    if (energy_last && !s->graph_e) {
        int rc = capture_step<T>(s, true, &s->graph_e, &s->graph_e_launches);
        if (rc) return rc;
    }
    CK(cudaEventRecord(s->ev_in, s->st));
    CK(cudaStreamWaitEvent(s->gst, s->ev_in, 0));
    for (int k = 0; k < plain; ++k) CK(cudaGraphLaunch(s->graph, s->gst));
    if (energy_last) CK(cudaGraphLaunch(s->graph_e, s->gst));
    CK(cudaEventRecord(s->ev_out, s->gst));
    CK(cudaStreamWaitEvent(s->st, s->ev_out, 0));
    s->launches += s->graph_launches * plain + (energy_last ? s->graph_e_launches : 0);
    return MISA_OK;
}

// after positions or velocities change outside a step: new forces (no
// kick) and the max speed that sets the next adaptive timestep
template <typename T>
int refresh(misa_sim *s, bool forces)
{
    MdArgs<T> m = md_args<T>(s);
    if (forces) {
        int rc = launch_forces<T>(s, 0, false);
        if (rc) return rc;
    }
    for (int r = 0; r < s->nrep; ++r) CK(cudaMemsetAsync(&s->sc[r].vmax_bits, 0, sizeof(unsigned long long), s->st));
    k_vmax<T><<<site_grid(s), 256, 0, s->st>>>(m);
    CK(cudaGetLastError());
    return MISA_OK;
}

// FP32 handles: whether the passes of tile shape k fit in the shared memory
// of a block -- the table window beside one staged tile (single-type passes;
// both alloy passes with several species); always true for FP64, whose
// tables stay in global memory
template <typename T>
bool shape_fits(const misa_sim *s, int k)
{
    if (sizeof(T) != 4) return true;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return false;
    const TileShape &t = kTiles[k];
    const int nwin = s->p.n_knots - 1 - seg_lo_of(s);
    const size_t tb = sizeof(float4) * (size_t)(nwin + 1);
    if (packed_smem_bytes(tb, t.tx, t.ty, t.tz, 1) > (size_t)optin) return false;
    if (s->dens_n3 && n3_smem_bytes(tb, t.tx, t.ty, t.tz, 1) > (size_t)optin) return false;
    if (s->nsp <= 1) return true;
    return alloy_smem_bytes(true, nwin, t.tx, t.ty, t.tz) <= (size_t)optin &&
           alloy_smem_bytes(false, nwin, t.tx, t.ty, t.tz) <= (size_t)optin;
}

// Tile autotuner: times the density pass and the force pass of the current
// state for every tile shape and keeps the fastest shape of each pass.
template <typename T>
int autotune(misa_sim *s)
{
    cudaEvent_t ev[3];
    for (auto &e : ev) CK(cudaEventCreate(&e));
    float best_d = 1e30f, best_f = 1e30f;
    int kd = 0, kf = 0;
    for (int k = 0; k < kNTiles; ++k) {
        if (!tile_ok(s->prec, kTiles[k]) || !shape_fits<T>(s, k)) continue;
        int rc = configure<T>(s, k, k);
        if (rc) return rc;
        rc = launch_forces<T>(s, 0, false);  // warm-up
        if (rc) return rc;
        GatherArgs<T> gd, gf;
        fill_gather<T>(s, gd, false);
        fill_gather<T>(s, gf, true);
        gd.kick = gf.kick = 0;
        CK(cudaEventRecord(ev[0], s->st));
        for (int q = 0; q < 3; ++q) launch_density<T>(s, gd, false);
        CK(cudaEventRecord(ev[1], s->st));
        for (int q = 0; q < 3; ++q) launch_force<T>(s, gf, false);
        CK(cudaEventRecord(ev[2], s->st));
        CK(cudaGetLastError());
        CK(cudaEventSynchronize(ev[2]));
        float md = 0.f, mf = 0.f;
        CK(cudaEventElapsedTime(&md, ev[0], ev[1]));
        CK(cudaEventElapsedTime(&mf, ev[1], ev[2]));
        if (md < best_d) {
            best_d = md;
            kd = k;
        }
        if (mf < best_f) {
            best_f = mf;
            kf = k;
        }
    }
    for (auto e : ev) cudaEventDestroy(e);
    return configure<T>(s, kd, kf);
}

template <typename T>
int create_impl(misa_sim *s)
{
    const long long ns = s->ns;
    const size_t capt = (size_t)s->cap * s->nrep;
    const int n = s->p.n_knots;
    size_t Tb = sizeof(T);
    s->reps_d = (RepDesc *)dalloc(s, sizeof(RepDesc) * s->nrep);
    s->sc = (DevScalars *)dalloc(s, sizeof(DevScalars) * s->nrep);
    // kick/drift: one block per kd_chunk sites of each replica, so that the
    // sweep's blocks carry equal work whatever the replicas' sizes
    s->kd_chunk = kKdChunkMax;
    while (s->kd_chunk > kKdChunkMin && s->ns / s->kd_chunk < 8LL * s->nsm) s->kd_chunk /= 2;
    s->kd_host.clear();
    for (int r = 0; r < s->nrep; ++r)
        for (long long b = 0; b < s->reps[r].ns; b += s->kd_chunk) s->kd_host.push_back(make_int2(r, (int)b));
    s->kd_blocks = (int)s->kd_host.size();
    s->kd_map = (int2 *)dalloc(s, sizeof(int2) * s->kd_host.size());
    if (!s->kd_map) return fail(s, MISA_EOOM, "device allocation failed (kick/drift map)");
    CK(cudaMemcpyAsync(s->kd_map, s->kd_host.data(), sizeof(int2) * s->kd_host.size(), cudaMemcpyHostToDevice,
                       s->st));
    s->tile_rep = (int *)dalloc(s, sizeof(int) * (size_t)s->ntile_cap);
    s->tile_flag = (int *)dalloc(s, sizeof(int) * (size_t)s->ntile_cap);
    s->reps_fd = (RepDesc *)dalloc(s, sizeof(RepDesc) * s->nrep);
    s->tile_rep_f = (int *)dalloc(s, sizeof(int) * (size_t)s->ntile_cap);
    s->tile_flag_f = (int *)dalloc(s, sizeof(int) * (size_t)s->ntile_cap);
    // a run-away is staged by at most 4 tiles per axis (7-cell window, tiles
    // of at least 4 cells, a partial last tile across the wrap)
    s->rt_cap = 64LL * s->cap * s->nrep;
    if (s->rt_cap > 0x7FFFFFFFLL) s->rt_cap = 0x7FFFFFFFLL;
    // counts and cursors of both maps in one block each (one memset per step)
    int *cnt2 = (int *)dalloc(s, sizeof(int) * (size_t)s->ntile_cap * 2);
    int *aux2 = (int *)dalloc(s, sizeof(int) * 4);
    if (!cnt2 || !aux2) return fail(s, MISA_EOOM, "device allocation failed (run-away tile index)");
    for (int k = 0; k < 2; ++k) {
        s->rt_cnt[k] = cnt2 + (size_t)k * s->ntile_cap;
        s->rt_aux[k] = aux2 + 2 * k;
        s->rt_off[k] = (int *)dalloc(s, sizeof(int) * (size_t)s->ntile_cap);
        s->rt_fill[k] = (int *)dalloc(s, sizeof(int) * (size_t)s->ntile_cap);
        s->rt_nz[k] = (int *)dalloc(s, sizeof(int) * (size_t)s->ntile_cap);
        s->rt_list[k] = (int *)dalloc(s, sizeof(int) * (size_t)s->rt_cap);
        if (!s->rt_off[k] || !s->rt_fill[k] || !s->rt_nz[k] || !s->rt_list[k])
            return fail(s, MISA_EOOM, "device allocation failed (run-away tile index)");
    }
    s->sid = (int *)dalloc(s, sizeof(int) * ns);
    s->claim = (int *)dalloc(s, sizeof(int) * ns);
    for (int d = 0; d < 3; ++d) {
        s->u[d] = (double *)dalloc(s, sizeof(double) * ns);
        s->v[d] = (double *)dalloc(s, sizeof(double) * ns);
        s->a[d] = dalloc(s, Tb * ns);
        s->s[d] = sizeof(T) == 8 ? (void *)s->u[d] : dalloc(s, Tb * ns);
        s->ra_u[d] = (double *)dalloc(s, sizeof(double) * capt);
        s->ra_v[d] = (double *)dalloc(s, sizeof(double) * capt);
        s->ra_s[d] = dalloc(s, Tb * capt);
        s->ra_a[d] = dalloc(s, Tb * capt);
        s->t_u[d] = (double *)dalloc(s, sizeof(double) * capt);
        s->t_v[d] = (double *)dalloc(s, sizeof(double) * capt);
        s->t_s[d] = dalloc(s, Tb * capt);
        s->t_a[d] = dalloc(s, Tb * capt);
        if (!s->u[d] || !s->v[d] || !s->a[d] || !s->s[d] || !s->ra_u[d] || !s->ra_v[d] || !s->ra_s[d] || !s->ra_a[d] ||
            !s->t_u[d] || !s->t_v[d] || !s->t_s[d] || !s->t_a[d])
            return fail(s, MISA_EOOM, "device allocation failed");
    }
    s->fp = dalloc(s, Tb * ns);
    s->rho = dalloc(s, Tb * ns);
    s->esite = (double *)dalloc(s, sizeof(double) * ns);
    if (sizeof(T) == 4) s->bmask = (unsigned long long *)dalloc(s, sizeof(unsigned long long) * ns);
    s->ra_home = (int *)dalloc(s, sizeof(int) * capt);
    s->ra_id = (int *)dalloc(s, sizeof(int) * capt);
    s->t_home = (int *)dalloc(s, sizeof(int) * capt);
    s->t_id = (int *)dalloc(s, sizeof(int) * capt);
    s->ra_fp = dalloc(s, Tb * capt);
    s->ra_rho = dalloc(s, Tb * capt);
    s->ra_e = (double *)dalloc(s, sizeof(double) * capt);
    s->knots = (double *)dalloc(s, sizeof(double) * 3 * n);
    s->tab_f = dalloc(s, sizeof(Vec4<T>) * n);
    s->tab_phi = dalloc(s, sizeof(Vec4<T>) * n);
    s->tab_F = dalloc(s, sizeof(Vec4<T>) * n);
    s->tab_d0 = dalloc(s, sizeof(Vec4<T>) * n);
    s->tab_d1 = dalloc(s, sizeof(Vec2<T>) * n);
    s->partial = (double *)dalloc(s, sizeof(double) * 512 * s->nrep);
    s->red_out = (double *)dalloc(s, sizeof(double) * 2 * s->nrep);
    s->out_buf = (double *)dalloc(s, sizeof(double) * 3 * ns);
    s->aux_int = (int *)dalloc(s, sizeof(int) * ns);
    s->aux_dbl = (double *)dalloc(s, sizeof(double) * 3 * ns);
    if (!s->reps_d || !s->sc || !s->tile_rep || !s->tile_flag || !s->reps_fd || !s->tile_rep_f || !s->tile_flag_f ||
        !s->sid || !s->claim || !s->fp || !s->rho ||
        !s->esite || (sizeof(T) == 4 && !s->bmask) || !s->ra_home || !s->ra_id || !s->t_home || !s->t_id || !s->ra_fp || !s->ra_rho || !s->ra_e ||
        !s->knots || !s->tab_f || !s->tab_phi || !s->tab_F || !s->tab_d0 || !s->tab_d1 || !s->partial ||
        !s->red_out || !s->out_buf || !s->aux_int || !s->aux_dbl)
        return fail(s, MISA_EOOM, "device allocation failed");
    CK(cudaMemcpyAsync(s->knots, s->fk.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->knots + n, s->pk.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->knots + 2 * n, s->Fk.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s->st));
    const double hr = s->p.rc / (n - 1), hrho = s->p.rho_max / (n - 1);
    k_spline_tables<T><<<(n + 255) / 256, 256, 0, s->st>>>(s->knots, s->knots + n, s->knots + 2 * n, n, hr, hrho,
                                                            (Vec4<T> *)s->tab_f, (Vec4<T> *)s->tab_phi,
                                                            (Vec4<T> *)s->tab_F, (Vec4<T> *)s->tab_d0,
                                                            (Vec2<T> *)s->tab_d1);
    if (sizeof(T) == 4) {
        void *ptrs[3] = {s->tab_f, s->tab_d0, s->tab_d1};
        const cudaChannelFormatDesc cd[3] = {cudaCreateChannelDesc<float4>(), cudaCreateChannelDesc<float4>(),
                                             cudaCreateChannelDesc<float2>()};
        const size_t bytes[3] = {sizeof(Vec4<T>) * (size_t)n, sizeof(Vec4<T>) * (size_t)n, sizeof(Vec2<T>) * (size_t)n};
        unsigned long long *out[3] = {&s->tex_f, &s->tex_d0, &s->tex_d1};
        for (int q = 0; q < 3; ++q) {
            cudaResourceDesc rd{};
            rd.resType = cudaResourceTypeLinear;
            rd.res.linear.devPtr = ptrs[q];
            rd.res.linear.desc = cd[q];
            rd.res.linear.sizeInBytes = bytes[q];
            cudaTextureDesc td{};
            td.readMode = cudaReadModeElementType;
            cudaTextureObject_t to = 0;
            CK(cudaCreateTextureObject(&to, &rd, &td, nullptr));
            *out[q] = to;
        }
    }
    // a fixed shape as asked (MISA_EINVAL if it does not fit); with the
    // autotuner the first built shape that fits starts
    int t0 = s->p.tile > 0 ? s->p.tile - 1 : 0;
    if (s->p.tile == 0)
        while (t0 + 1 < kNTiles && (!tile_ok(s->prec, kTiles[t0]) || !shape_fits<T>(s, t0))) ++t0;
    int rc = configure<T>(s, t0, t0);
    if (rc) return rc;
    MdArgs<T> m = md_args<T>(s);
    k_init_crystal<T><<<site_grid(s), 256, 0, s->st>>>(m);
    s->ra_index_valid = false;
    CK(cudaGetLastError());
    if (s->p.tile == 0) {
        rc = autotune<T>(s);
        if (rc) return rc;
    }
    return refresh<T>(s, true);
}

// Sets the state from device arrays xd (3 natoms) and vd (3 natoms or
// null); xd may be out_buf (each atom's displacement from its nearest site
// then overwrites its position in place).  done, if given, is recorded once
// xd and vd have been read.
template <typename T>
int set_state_dev(misa_sim *s, const double *xd, const double *vd, cudaEvent_t done)
{
    const long long N = s->ns;
    MdArgs<T> m = md_args<T>(s);
    s->ra_index_valid = false;
    k_reset_list<T><<<rep_blocks(s), 128, 0, s->st>>>(m);
    k_clear_sites<T><<<site_grid(s), 256, 0, s->st>>>(m);
    k_state_claim<T><<<site_grid(s), 256, 0, s->st>>>(m, xd, s->aux_int, s->out_buf);
    if (!vd) {
        CK(cudaMemsetAsync(s->v[0], 0, sizeof(double) * N, s->st));
        CK(cudaMemsetAsync(s->v[1], 0, sizeof(double) * N, s->st));
        CK(cudaMemsetAsync(s->v[2], 0, sizeof(double) * N, s->st));
    }
    k_state_place<T><<<site_grid(s), 256, 0, s->st>>>(m, vd, s->aux_int, s->out_buf);
    if (done) CK(cudaEventRecord(done, s->st));
    k_ra_sort<T><<<s->nrep, 1024, sizeof(unsigned long long) * kSortMax, s->st>>>(m);
    CK(cudaGetLastError());
    return refresh<T>(s, true);
}

template <typename T>
int set_state_impl(misa_sim *s, const double *x, const double *v)
{
    const long long N = s->ns;
    CK(cudaMemcpyAsync(s->out_buf, x, sizeof(double) * 3 * N, cudaMemcpyDefault, s->st));
    const double *vd = nullptr;
    if (v) {
        CK(cudaMemcpyAsync(s->aux_dbl, v, sizeof(double) * 3 * N, cudaMemcpyDefault, s->st));
        vd = s->aux_dbl;
    }
    return set_state_dev<T>(s, s->out_buf, vd, nullptr);
}

// per-replica potential and kinetic energy (eV) into pe[r], ke[r]
template <typename T>
int reduce_energy(misa_sim *s, double *pe, double *ke, double *per_atom)
{
    // per-atom energies of the current positions: from the last step when
    // it evaluated them (misa_step_energies), else one evaluation now
    if (!s->energy_valid) {
        int rc = launch_forces<T>(s, 0, true);
        if (rc) return rc;
        s->energy_valid = true;
    }
    MdArgs<T> m = md_args<T>(s);
    const int nb = red_blocks(s);
    k_sum_stage1<T><<<dim3(nb, s->nrep), 256, 0, s->st>>>(m, 0, s->partial);
    k_sum_stage2<<<s->nrep, 1024, 0, s->st>>>(s->partial, nb, s->red_out);
    k_sum_stage1<T><<<dim3(nb, s->nrep), 256, 0, s->st>>>(m, 1, s->partial);
    k_sum_stage2<<<s->nrep, 1024, 0, s->st>>>(s->partial, nb, s->red_out + s->nrep);
    if (per_atom) {
        k_scatter<T><<<site_grid(s), 256, 0, s->st>>>(m, 4, s->out_buf);
        CK(cudaMemcpyAsync(per_atom, s->out_buf, sizeof(double) * s->ns, cudaMemcpyDefault, s->st));
    }
    std::vector<double> h(2 * s->nrep);
    CK(cudaMemcpyAsync(h.data(), s->red_out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    for (int r = 0; r < s->nrep; ++r) {
        if (pe) pe[r] = h[r];
        if (ke) ke[r] = 0.5 * s->p.mass * h[s->nrep + r] / kAccUnit;
    }
    return MISA_OK;
}

template <typename T>
int scatter_out(misa_sim *s, int kind, double *out)
{
    MdArgs<T> m = md_args<T>(s);
    if (kind == 3) {
        int rc = launch_forces<T>(s, 0, true);
        if (rc) return rc;
    }
    k_scatter<T><<<site_grid(s), 256, 0, s->st>>>(m, kind, s->out_buf);
    CK(cudaGetLastError());
    size_t cnt = kind >= 3 ? (size_t)s->ns : 3 * (size_t)s->ns;
    CK(cudaMemcpyAsync(out, s->out_buf, sizeof(double) * cnt, cudaMemcpyDefault, s->st));
    CK(cudaStreamSynchronize(s->st));
    return MISA_OK;
}

// E_i of the current positions into e_buf (handle's stream), then copied to
// out on the output stream; nothing waits on the host
template <typename T>
int energies_async(misa_sim *s, double *out)
{
    if (!s->ost) {
        CK(cudaStreamCreateWithFlags(&s->ost, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&s->ev_e_ready, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&s->ev_e_done, cudaEventDisableTiming));
    }
    if (!s->e_buf) {
        s->e_buf = (double *)dalloc(s, sizeof(double) * (size_t)s->ns);
        if (!s->e_buf) return fail(s, MISA_EOOM, "get_energies_async: output buffer");
    }
    if (!s->energy_valid) {
        int rc = launch_forces<T>(s, 0, true);
        if (rc) return rc;
        s->energy_valid = true;
    }
    // the previous copy out of e_buf is complete before it is overwritten
    CK(cudaStreamWaitEvent(s->st, s->ev_e_done, 0));
    MdArgs<T> m = md_args<T>(s);
    k_scatter<T><<<site_grid(s), 256, 0, s->st>>>(m, 4, s->e_buf);
    CK(cudaGetLastError());
    s->launches += 1;
    CK(cudaEventRecord(s->ev_e_ready, s->st));
    CK(cudaStreamWaitEvent(s->ost, s->ev_e_ready, 0));
    CK(cudaMemcpyAsync(out, s->e_buf, sizeof(double) * (size_t)s->ns, cudaMemcpyDefault, s->ost));
    CK(cudaEventRecord(s->ev_e_done, s->ost));
    return MISA_OK;
}

int check_status(misa_sim *s)
{
    unsigned st = 0;
    CK(cudaMemcpyAsync(&st, &s->sc[0].status, sizeof(unsigned), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    if (st & kStRunawayOverflow) return fail(s, MISA_ERUNAWAY_OVERFLOW, "run-away list overflow");
    if (st & kStNonfinite) return fail(s, MISA_EUNSTABLE, "non-finite force or velocity");
    return MISA_OK;
}

int validate(const misa_params &p, misa_sim *s)
{
    if (!(p.a0 > 0) || !(p.mass > 0) || !(p.rc > 0) || !(p.skin > 0)) return fail(s, MISA_EINVAL, "a0, mass, rc, skin must be > 0");
    if (p.n_knots < 8 || !p.f_knots || !p.phi_knots || !p.F_knots || !(p.rho_max > 0))
        return fail(s, MISA_EINVAL, "three knot tables (n >= 8) and rho_max > 0 are required");
    double half = 0.5 * p.a0, roff = (p.rc + 2.0 * p.skin) / half;
    if (roff * roff >= 27.0) return fail(s, MISA_EINVAL, "(rc + 2 skin) must be below sqrt(27) a0/2 (2-cell halo)");
    if (p.skin >= 0.25 * std::sqrt(3.0) * p.a0) return fail(s, MISA_EINVAL, "skin must be below half the nearest-neighbour distance");
    if (p.precision != MISA_FP64 && p.precision != MISA_FP32_FORCE) return fail(s, MISA_EINVAL, "precision");
    if (!(p.dt_max > 0) || p.dx_max < 0) return fail(s, MISA_EINVAL, "dt_max > 0, dx_max >= 0");
    if (!!p.alloc != !!p.free) return fail(s, MISA_EINVAL, "alloc and free hooks come together");
    if (p.tile < 0 || p.tile > kNTiles) return fail(s, MISA_EINVAL, "tile index");
    if (p.tile > 0 && !tile_ok(p.precision, kTiles[p.tile - 1])) return fail(s, MISA_EINVAL, "tile shape not built for this precision");
    return MISA_OK;
}

// builds the host side of a batch (replica table, knots); no device work
int init_host(misa_sim *s, const misa_params &p, int nrep, const int32_t *dims)
{
    s->p = p;
    s->fk.assign(p.f_knots, p.f_knots + p.n_knots);
    s->pk.assign(p.phi_knots, p.phi_knots + p.n_knots);
    s->Fk.assign(p.F_knots, p.F_knots + p.n_knots);
    s->p.f_knots = s->fk.data();
    s->p.phi_knots = s->pk.data();
    s->p.F_knots = s->Fk.data();
    s->prec = p.precision;
    s->nrep = nrep;
    s->dims.assign(dims, dims + 3 * nrep);
    long long ns = 0, maxns = 0;
    for (int r = 0; r < nrep; ++r) {
        const int nx = dims[3 * r], ny = dims[3 * r + 1], nz = dims[3 * r + 2];
        if (nx < 6 || ny < 6 || nz < 6) return fail(s, MISA_EINVAL, "each box dimension must be >= 6 cells");
        long long n = 2LL * nx * ny * nz;
        maxns = n > maxns ? n : maxns;
        ns += n;
    }
    if (ns >= (1LL << 31)) return fail(s, MISA_EINVAL, "too many atoms for 32-bit ids");
    s->ns = ns;
    long long cap = p.runaway_capacity > 0 ? p.runaway_capacity : (maxns / 64 > 4096 ? maxns / 64 : 4096);
    if (cap > kSortMax) cap = kSortMax;
    s->cap = (int)cap;
    s->reps.resize(nrep);
    long long base = 0;
    long long tcap = 0;
    for (int r = 0; r < nrep; ++r) {
        RepDesc &rd = s->reps[r];
        std::memset(&rd, 0, sizeof(rd));
        rd.nx = dims[3 * r];
        rd.ny = dims[3 * r + 1];
        rd.nz = dims[3 * r + 2];
        rd.site_base = base;
        rd.ns = 2LL * rd.nx * rd.ny * rd.nz;
        rd.ra_base = r * s->cap;
        rd.cap = s->cap;
        base += rd.ns;
        long long worst = 0;
        for (int k = 0; k < kNTiles; ++k) {
            long long nt = (long long)((rd.nx + kTiles[k].tx - 1) / kTiles[k].tx) * ((rd.ny + kTiles[k].ty - 1) / kTiles[k].ty) *
                           ((rd.nz + kTiles[k].tz - 1) / kTiles[k].tz);
            worst = nt > worst ? nt : worst;
        }
        tcap += worst;
    }
    s->ntile_cap = tcap;
    return MISA_OK;
}

int stats_of(misa_sim *s, int r, const DevScalars &h, unsigned status, misa_stats *o)
{
    o->step = h.step;
    o->time = h.t;
    double vmax;
    std::memcpy(&vmax, &h.vmax_bits, sizeof(double));
    o->vmax = vmax;
    double dt = s->p.dt_max;
    if (s->p.dx_max > 0 && vmax > 0) dt = std::fmin(s->p.dt_max, s->p.dx_max / vmax);
    o->dt = dt;
    o->natoms = r < 0 ? s->ns : s->reps[r].ns;
    o->nsites = o->natoms;
    o->n_runaway = h.n_ra;
    o->n_vacant = h.n_ra;
    o->status = status;
    o->launches = s->launches;
    return MISA_OK;
}

// New knot values for the three tables (same n and grids); the forces of
// the current positions are re-evaluated.
template <typename T>
int set_tables_impl(misa_sim *s, const double *f, const double *phi, const double *F)
{
    const int n = s->p.n_knots;
    CK(cudaMemcpyAsync(s->knots, f, sizeof(double) * n, cudaMemcpyDefault, s->st));
    CK(cudaMemcpyAsync(s->knots + n, phi, sizeof(double) * n, cudaMemcpyDefault, s->st));
    CK(cudaMemcpyAsync(s->knots + 2 * n, F, sizeof(double) * n, cudaMemcpyDefault, s->st));
    const double hr = s->p.rc / (n - 1), hrho = s->p.rho_max / (n - 1);
    k_spline_tables<T><<<(n + 255) / 256, 256, 0, s->st>>>(s->knots, s->knots + n, s->knots + 2 * n, n, hr, hrho,
                                                            (Vec4<T> *)s->tab_f, (Vec4<T> *)s->tab_phi,
                                                            (Vec4<T> *)s->tab_F, (Vec4<T> *)s->tab_d0,
                                                            (Vec2<T> *)s->tab_d1);
    CK(cudaGetLastError());
    if (s->nsp != 1) drop_graphs(s);  // back to the single-type passes
    s->nsp = 1;
    return refresh<T>(s, true);
}

// Alloy tables and per-atom species (Eq. eam_base with atom types).  One
// species falls back to the single-type tables and gathers.
template <typename T>
int set_species_impl(misa_sim *s, int nsp, const double *f, const double *F, const double *phi, const int8_t *types)
{
    const int n = s->p.n_knots;
    if (nsp == 1) {
        std::vector<double> pf(n), pF(n), pp(n);
        CK(cudaMemcpy(pf.data(), f, sizeof(double) * n, cudaMemcpyDefault));
        CK(cudaMemcpy(pF.data(), F, sizeof(double) * n, cudaMemcpyDefault));
        CK(cudaMemcpy(pp.data(), phi, sizeof(double) * n, cudaMemcpyDefault));
        s->nsp = 1;
        drop_graphs(s);
        return set_tables_impl<T>(s, pf.data(), pp.data(), pF.data());
    }
    std::vector<int8_t> ht((size_t)s->ns);
    CK(cudaMemcpy(ht.data(), types, (size_t)s->ns, cudaMemcpyDefault));
    std::vector<long long> cnt(nsp, 0);
    for (int8_t t : ht) {
        if (t < 0 || t >= nsp) return fail(s, MISA_EINVAL, "atom type outside [0, n_species)");
        ++cnt[t];
    }
    int maj = 0;
    for (int t = 1; t < nsp; ++t)
        if (cnt[t] > cnt[maj]) maj = t;
    const int npair = nsp * (nsp + 1) / 2;
    if (nsp > s->al_cap) {
        const int cp = kMaxSpecies, pp = kMaxSpecies * (kMaxSpecies + 1) / 2;
        if (!s->atype) s->atype = (int8_t *)dalloc(s, (size_t)s->ns);
        s->al_knots = (double *)dalloc(s, sizeof(double) * (size_t)n * (2 * cp + pp));
        s->al_fv = dalloc(s, sizeof(Vec4<T>) * (size_t)n * cp);
        s->al_fd = dalloc(s, sizeof(Vec4<T>) * (size_t)n * cp);
        s->al_Fv = dalloc(s, sizeof(Vec4<T>) * (size_t)n * cp);
        s->al_pv = dalloc(s, sizeof(Vec4<T>) * (size_t)n * pp);
        s->al_pd = dalloc(s, sizeof(Vec4<T>) * (size_t)n * pp);
        if (!s->atype || !s->al_knots || !s->al_fv || !s->al_fd || !s->al_Fv || !s->al_pv || !s->al_pd)
            return fail(s, MISA_EOOM, "alloy tables");
        s->al_cap = cp;
    }
    CK(cudaMemcpyAsync(s->atype, ht.data(), (size_t)s->ns, cudaMemcpyHostToDevice, s->st));
    double *kf = s->al_knots, *kF = kf + (size_t)nsp * n, *kp = kF + (size_t)nsp * n;
    CK(cudaMemcpyAsync(kf, f, sizeof(double) * (size_t)nsp * n, cudaMemcpyDefault, s->st));
    CK(cudaMemcpyAsync(kF, F, sizeof(double) * (size_t)nsp * n, cudaMemcpyDefault, s->st));
    CK(cudaMemcpyAsync(kp, phi, sizeof(double) * (size_t)npair * n, cudaMemcpyDefault, s->st));
    const double hr = s->p.rc / (n - 1), hrho = s->p.rho_max / (n - 1);
    k_alloy_tables<T><<<256, 256, 0, s->st>>>(kf, kF, kp, nsp, npair, n, hr, hrho, (Vec4<T> *)s->al_fv,
                                              (Vec4<T> *)s->al_fd, (Vec4<T> *)s->al_Fv, (Vec4<T> *)s->al_pv,
                                              (Vec4<T> *)s->al_pd);
    CK(cudaGetLastError());
    if (sizeof(T) == 4) {  // texture objects over the tables of the FP32 alloy gathers
        for (unsigned long long *t : {&s->tex_afv, &s->tex_afd, &s->tex_apd}) {
            if (*t) cudaDestroyTextureObject((cudaTextureObject_t)*t);
            *t = 0;
        }
        void *ptrs[3] = {s->al_fv, s->al_fd, s->al_pd};
        const size_t cnt[3] = {(size_t)nsp * n, (size_t)nsp * n, (size_t)npair * n};
        unsigned long long *out[3] = {&s->tex_afv, &s->tex_afd, &s->tex_apd};
        for (int q = 0; q < 3; ++q) {
            cudaResourceDesc rd{};
            rd.resType = cudaResourceTypeLinear;
            rd.res.linear.devPtr = ptrs[q];
            rd.res.linear.desc = cudaCreateChannelDesc<float4>();
            rd.res.linear.sizeInBytes = sizeof(float4) * cnt[q];
            cudaTextureDesc td{};
            td.readMode = cudaReadModeElementType;
            cudaTextureObject_t to = 0;
            CK(cudaCreateTextureObject(&to, &rd, &td, nullptr));
            *out[q] = to;
        }
    }
    CK(cudaStreamSynchronize(s->st));  // ht is a host temporary
    s->nsp = nsp;
    s->amaj = maj;
    if (!shape_fits<T>(s, s->tile) || !shape_fits<T>(s, s->tile_f)) {
        // the current shapes' alloy passes do not fit: the first shape that does
        int k = 0;
        while (k < kNTiles && (!tile_ok(s->prec, kTiles[k]) || !shape_fits<T>(s, k))) ++k;
        if (k == kNTiles) return fail(s, MISA_EINVAL, "no tile shape fits the alloy passes' shared memory");
        int rc = configure<T>(s, k, k);
        if (rc) return rc;
    } else {
        int rc = configure<T>(s, s->tile, s->tile_f);  // the alloy passes' kernel attributes
        if (rc) return rc;
    }
    drop_graphs(s);
    int rc = refresh<T>(s, true);
    if (rc) return rc;
    return check_status(s);
}

// Loss and knot gradient of the current state against target forces and
// energies (Fref: 3 natoms, Eref: nrep); see misa_adjoint.cuh.
template <typename T>
int loss_grad_impl(misa_sim *s, const double *Fref, const double *Eref, double *loss, double *grad)
{
    if (s->nsp > 1) return fail(s, MISA_EINVAL, "the knot gradient is built for one atom type");
    const int n = s->p.n_knots;
    const size_t capt = (size_t)s->cap * s->nrep;
    // FP32: two bin copies per CTA when they fit, else one
    const size_t bin_bytes = sizeof(T) * 5 * (size_t)n;
    const int copies = sizeof(T) == 4 && 2 * bin_bytes <= 227u * 1024u ? 2 : 1;
    if (bin_bytes > 227u * 1024u) return fail(s, MISA_EINVAL, "too many knots for the gradient bins");
    if (!s->dl) {
        for (int d = 0; d < 3; ++d) {
            s->lam[d] = dalloc(s, sizeof(T) * s->ns);
            s->ra_lam[d] = dalloc(s, sizeof(T) * capt);
            if (!s->lam[d] || !s->ra_lam[d]) return fail(s, MISA_EOOM, "adjoint work arrays");
        }
        s->dl = dalloc(s, sizeof(T) * s->ns);
        s->cw = dalloc(s, sizeof(T) * s->ns);
        s->ra_dl = dalloc(s, sizeof(T) * capt);
        // FP32: one 1024-thread CTA per SM (two bin copies); FP64: two 256-thread CTAs
        int gx = ((sizeof(T) == 4 ? s->nsm : s->nsm * 2) + s->nrep - 1) / s->nrep;
        s->adj_cta = gx < 1 ? 1 : gx;
        s->adj_partial = (double *)dalloc(s, sizeof(double) * 5 * n * (size_t)s->adj_cta * s->nrep);
        s->adj_sum = (double *)dalloc(s, sizeof(double) * 5 * n);
        s->adj_grad = (double *)dalloc(s, sizeof(double) * 3 * n);
        s->adj_eref = (double *)dalloc(s, sizeof(double) * s->nrep * 2);
        s->adj_fref = (double *)dalloc(s, sizeof(double) * 3 * s->ns);
        if (!s->dl || !s->cw || !s->ra_dl || !s->adj_partial || !s->adj_sum || !s->adj_grad || !s->adj_eref ||
            !s->adj_fref)
            return fail(s, MISA_EOOM, "adjoint work arrays");
        CK(cudaFuncSetAttribute(k_adj_grad<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bin_bytes * copies)));
    }
    // forward: rho, F', E_i, forces of the current positions
    int rc = launch_forces<T>(s, 0, true);
    if (rc) return rc;
    MdArgs<T> m = md_args<T>(s);
    const int nb = red_blocks(s);
    k_sum_stage1<T><<<dim3(nb, s->nrep), 256, 0, s->st>>>(m, 0, s->partial);
    k_sum_stage2<<<s->nrep, 1024, 0, s->st>>>(s->partial, nb, s->red_out);  // E_r
    CK(cudaMemcpyAsync(s->adj_fref, Fref, sizeof(double) * 3 * s->ns, cudaMemcpyDefault, s->st));
    CK(cudaMemcpyAsync(s->adj_eref, Eref, sizeof(double) * s->nrep, cudaMemcpyDefault, s->st));
    AdjArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.reps = s->reps_d;
    a.nrep = s->nrep;
    a.sid = s->sid;
    a.ux = (const T *)s->s[0]; a.uy = (const T *)s->s[1]; a.uz = (const T *)s->s[2];
    a.fp = (const T *)s->fp; a.rho = (const T *)s->rho;
    a.ax = (const T *)s->a[0]; a.ay = (const T *)s->a[1]; a.az = (const T *)s->a[2];
    a.ra_home = s->ra_home; a.ra_id = s->ra_id;
    a.ra_ux = (const T *)s->ra_s[0]; a.ra_uy = (const T *)s->ra_s[1]; a.ra_uz = (const T *)s->ra_s[2];
    a.ra_fp = (const T *)s->ra_fp; a.ra_rho = (const T *)s->ra_rho;
    a.ra_ax = (const T *)s->ra_a[0]; a.ra_ay = (const T *)s->ra_a[1]; a.ra_az = (const T *)s->ra_a[2];
    a.sc = s->sc;
    a.tab_d0 = (const Vec4<T> *)s->tab_d0;
    a.tab_F = (const Vec4<T> *)s->tab_F;
    a.n = n;
    const double half = 0.5 * s->p.a0;
    a.half = (T)half;
    a.hr = (T)(s->p.rc / (n - 1));
    a.hrho = (T)(s->p.rho_max / (n - 1));
    a.inv_hr = (T)((n - 1) / s->p.rc);
    a.inv_hrho = (T)((n - 1) / s->p.rho_max);
    a.S = (T)(half / (s->p.rc / (n - 1)));
    fill_split(a.split, half / (s->p.rc / (n - 1)));
    a.rho_max = (T)s->p.rho_max;
    const double rcl = s->p.rc / half;
    a.rc2 = (T)(rcl * rcl);
    a.rfloor2 = (T)((kRfloor / half) * (kRfloor / half));
    a.acc_conv = kAccUnit / s->p.mass;
    a.inv_acc_conv = s->p.mass / kAccUnit;
    a.Fref = s->adj_fref;
    a.Eref = s->adj_eref;
    a.Etot = s->red_out;
    a.lam_x = (T *)s->lam[0]; a.lam_y = (T *)s->lam[1]; a.lam_z = (T *)s->lam[2];
    a.ra_lx = (T *)s->ra_lam[0]; a.ra_ly = (T *)s->ra_lam[1]; a.ra_lz = (T *)s->ra_lam[2];
    a.dl = (T *)s->dl; a.ra_dl = (T *)s->ra_dl; a.cw = (T *)s->cw;
    const double roff = (s->p.rc + 2.0 * s->p.skin) / half;
    int nsh = 0;
    while (nsh < kLVec.nshell && kLVec.shell_n2[nsh] <= roff * roff) ++nsh;
    a.nvec = kLVec.shell_begin[nsh];
    // the per-tile run-away index of the density map that the forward pass
    // built (the list does not change during the evaluation): sites and
    // run-aways scan only the run-aways within reach, in list order
    a.tile_flag = s->tile_flag;
    a.tx = kTiles[s->tile].tx; a.ty = kTiles[s->tile].ty; a.tz = kTiles[s->tile].tz;
    a.ra_toff = s->rt_off[0]; a.ra_tcnt = s->rt_cnt[0]; a.ra_tlist = s->rt_list[0];
    k_adj_lambda<T><<<dim3(nb, s->nrep), 256, 0, s->st>>>(a, s->partial);
    k_sum_stage2<<<s->nrep, 1024, 0, s->st>>>(s->partial, nb, s->red_out + s->nrep);  // sum |F - Fref|^2
    k_adj_dl<T><<<site_grid(s), 256, 0, s->st>>>(a);
    k_adj_grad<T><<<dim3(s->adj_cta, s->nrep), kGradThreads<T>, bin_bytes * copies, s->st>>>(a, s->adj_partial,
                                                                                             copies);
    k_adj_reduce<<<(5 * n + 31) / 32, dim3(32, 8), 0, s->st>>>(s->adj_partial, s->adj_cta * s->nrep, 5 * n, s->adj_sum);
    k_adj_stencil<<<(3 * n + 255) / 256, 256, 0, s->st>>>(s->adj_sum, n, s->adj_grad);
    s->launches += 9;
    CK(cudaGetLastError());
    if (grad) CK(cudaMemcpyAsync(grad, s->adj_grad, sizeof(double) * 3 * n, cudaMemcpyDefault, s->st));
    std::vector<double> h(2 * s->nrep), er(s->nrep);
    CK(cudaMemcpyAsync(h.data(), s->red_out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(er.data(), s->adj_eref, sizeof(double) * s->nrep, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    double L = 0.0;
    for (int r = 0; r < s->nrep; ++r) {
        const double N = (double)s->reps[r].ns;
        const double de = (h[r] - er[r]) / N;
        L += h[s->nrep + r] / (3.0 * N) + de * de;
    }
    if (loss) *loss = L;
    return MISA_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

void misa_default_params(misa_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->nx = p->ny = p->nz = 10;
    p->a0 = 2.855;
    p->mass = 55.845;
    p->rc = 5.6;
    p->skin = 0.6;
    p->n_knots = 0;
    p->precision = MISA_FP32_FORCE;
    p->reassign_period = 10;
    p->dt_max = 1.0;
    p->dx_max = 0.0;
    p->runaway_capacity = 0;
    p->tile = 0;
}

int misa_create_batch(const misa_params *pp, int32_t nrep, const int32_t *dims, void *stream, misa_sim **out)
{
    misa_sim *none = nullptr;
    if (!pp || !out || nrep < 1 || !dims) return fail(none, MISA_EINVAL, "null argument or nrep < 1");
    *out = nullptr;
    int rc = validate(*pp, none);
    if (rc) return rc;
    misa_sim *s = new misa_sim();
    rc = init_host(s, *pp, nrep, dims);
    if (rc) {
        g_create_error = s->err;
        delete s;
        return rc;
    }
    s->st = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (s->nsm <= 0) s->nsm = 1;
    if (cudaStreamCreateWithFlags(&s->gst, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming) != cudaSuccess)
        rc = fail(s, MISA_ECUDA, "stream/event creation failed");
    if (!rc) rc = s->prec == MISA_FP64 ? create_impl<double>(s) : create_impl<float>(s);
    if (rc == MISA_OK) {
        cudaError_t e = cudaStreamSynchronize(s->st);
        if (e != cudaSuccess) rc = fail(s, MISA_ECUDA, std::string("create: ") + cudaGetErrorString(e));
    }
    if (rc != MISA_OK) {
        g_create_error = s->err;
        misa_destroy(s);
        return rc;
    }
    *out = s;
    return MISA_OK;
}

int misa_create(const misa_params *pp, void *stream, misa_sim **out)
{
    if (!pp) return fail(nullptr, MISA_EINVAL, "null argument");
    const int32_t dims[3] = {pp->nx, pp->ny, pp->nz};
    return misa_create_batch(pp, 1, dims, stream, out);
}

void misa_destroy(misa_sim *s)
{
    if (!s) return;
    cudaStreamSynchronize(s->st);
    if (s->gst) cudaStreamSynchronize(s->gst);
    if (s->cst) cudaStreamSynchronize(s->cst);
    drop_graphs(s);
    for (unsigned long long t : {s->tex_f, s->tex_d0, s->tex_d1, s->tex_afv, s->tex_afd, s->tex_apd})
        if (t) cudaDestroyTextureObject((cudaTextureObject_t)t);
    for (auto e : s->ev_pool) cudaEventDestroy(e);
    if (s->ev_in) cudaEventDestroy(s->ev_in);
    if (s->ev_out) cudaEventDestroy(s->ev_out);
    if (s->gst) cudaStreamDestroy(s->gst);
    if (s->ev_stg) cudaEventDestroy(s->ev_stg);
    if (s->ev_stg_free) cudaEventDestroy(s->ev_stg_free);
    if (s->cst) cudaStreamDestroy(s->cst);
    if (s->ost) cudaStreamSynchronize(s->ost);
    if (s->ev_e_ready) cudaEventDestroy(s->ev_e_ready);
    if (s->ev_e_done) cudaEventDestroy(s->ev_e_done);
    if (s->ost) cudaStreamDestroy(s->ost);
    for (auto &a : s->allocs) {
        if (s->p.free) s->p.free(a.first, a.second, s->p.alloc_ctx);
        else cudaFree(a.first);
    }
    delete s;
}

const char *misa_last_error(const misa_sim *s) { return s ? s->err.c_str() : g_create_error.c_str(); }

int misa_replica_count(const misa_sim *s) { return s ? s->nrep : 0; }

int misa_replica_info(const misa_sim *s, int32_t r, int32_t dims[3], int64_t *atom_base, int64_t *natoms)
{
    if (!s || r < 0 || r >= s->nrep) return MISA_EINVAL;
    if (dims) {
        dims[0] = s->reps[r].nx;
        dims[1] = s->reps[r].ny;
        dims[2] = s->reps[r].nz;
    }
    if (atom_base) *atom_base = s->reps[r].site_base;
    if (natoms) *natoms = s->reps[r].ns;
    return MISA_OK;
}

int misa_set_state(misa_sim *s, const double *x, const double *v, int64_t n)
{
    if (s) s->energy_valid = false;
    if (!s) return MISA_EINVAL;
    if (!x || n != s->ns) return fail(s, MISA_EINVAL, "set_state: x required, n must equal natoms");
    return s->prec == MISA_FP64 ? set_state_impl<double>(s, x, v) : set_state_impl<float>(s, x, v);
}

int misa_stage_state(misa_sim *s, const double *x, const double *v, int64_t n)
{
    if (!s) return MISA_EINVAL;
    if (!x || n != s->ns) return fail(s, MISA_EINVAL, "stage_state: x required, n must equal natoms");
    if (!s->cst) {
        CK(cudaStreamCreateWithFlags(&s->cst, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&s->ev_stg, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&s->ev_stg_free, cudaEventDisableTiming));
    }
    if (!s->stg_x) {
        s->stg_x = (double *)dalloc(s, sizeof(double) * 3 * s->ns);
        if (!s->stg_x) return fail(s, MISA_EOOM, "stage_state: staging buffer");
    }
    if (v && !s->stg_v) {
        s->stg_v = (double *)dalloc(s, sizeof(double) * 3 * s->ns);
        if (!s->stg_v) return fail(s, MISA_EOOM, "stage_state: staging buffer");
    }
    // the previous staged copy is complete before this call returns (its
    // host arrays may then be released); the new copies wait on the device
    // until the previous staged state has been read
    CK(cudaEventSynchronize(s->ev_stg));
    CK(cudaStreamWaitEvent(s->cst, s->ev_stg_free, 0));
    CK(cudaMemcpyAsync(s->stg_x, x, sizeof(double) * 3 * s->ns, cudaMemcpyDefault, s->cst));
    if (v) CK(cudaMemcpyAsync(s->stg_v, v, sizeof(double) * 3 * s->ns, cudaMemcpyDefault, s->cst));
    CK(cudaEventRecord(s->ev_stg, s->cst));
    s->stg_pending = true;
    s->stg_has_v = v != nullptr;
    return MISA_OK;
}

int misa_set_state_staged(misa_sim *s)
{
    if (s) s->energy_valid = false;
    if (!s) return MISA_EINVAL;
    if (!s->stg_pending) return fail(s, MISA_EINVAL, "set_state_staged: no state staged");
    CK(cudaStreamWaitEvent(s->st, s->ev_stg, 0));
    s->stg_pending = false;
    const double *vd = s->stg_has_v ? s->stg_v : nullptr;
    return s->prec == MISA_FP64 ? set_state_dev<double>(s, s->stg_x, vd, s->ev_stg_free)
                                : set_state_dev<float>(s, s->stg_x, vd, s->ev_stg_free);
}

int misa_set_velocities(misa_sim *s, const double *v, int64_t n)
{
    if (!s) return MISA_EINVAL;
    if (!v || n != s->ns) return fail(s, MISA_EINVAL, "set_velocities: n must equal natoms");
    CK(cudaMemcpyAsync(s->aux_dbl, v, sizeof(double) * 3 * s->ns, cudaMemcpyDefault, s->st));
    if (s->prec == MISA_FP64) {
        k_set_velocities<double><<<site_grid(s), 256, 0, s->st>>>(md_args<double>(s), s->aux_dbl);
        return refresh<double>(s, false);
    }
    k_set_velocities<float><<<site_grid(s), 256, 0, s->st>>>(md_args<float>(s), s->aux_dbl);
    return refresh<float>(s, false);
}

int misa_insert_pka(misa_sim *s, int64_t atom, double energy, const double dir[3])
{
    if (!s) return MISA_EINVAL;
    if (!dir || !(energy >= 0)) return fail(s, MISA_EINVAL, "insert_pka: bad direction or energy");
    double nrm = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    if (!(nrm > 0)) return fail(s, MISA_EINVAL, "insert_pka: zero direction");
    if (atom < 0) {
        const RepDesc &rd = s->reps[0];
        atom = rd.site_base + 2LL * (((long long)(rd.nz / 2) * rd.ny + rd.ny / 2) * rd.nx + rd.nx / 2);
    }
    if (atom >= s->ns) return fail(s, MISA_EINVAL, "insert_pka: atom id out of range");
    double speed = std::sqrt(2.0 * energy / s->p.mass * kAccUnit);
    double vx = speed * dir[0] / nrm, vy = speed * dir[1] / nrm, vz = speed * dir[2] / nrm;
    if (s->prec == MISA_FP64) {
        k_pka<double><<<site_grid(s), 256, 0, s->st>>>(md_args<double>(s), (int)atom, vx, vy, vz);
        return refresh<double>(s, false);
    }
    k_pka<float><<<site_grid(s), 256, 0, s->st>>>(md_args<float>(s), (int)atom, vx, vy, vz);
    return refresh<float>(s, false);
}

int misa_insert_pka_replica(misa_sim *s, int32_t r, double energy, const double dir[3])
{
    if (!s) return MISA_EINVAL;
    if (r < 0 || r >= s->nrep) return fail(s, MISA_EINVAL, "insert_pka_replica: replica out of range");
    const RepDesc &rd = s->reps[r];
    long long atom = rd.site_base + 2LL * (((long long)(rd.nz / 2) * rd.ny + rd.ny / 2) * rd.nx + rd.nx / 2);
    return misa_insert_pka(s, atom, energy, dir);
}

static int step_impl(misa_sim *s, int n, bool energy_last)
{
    if (!s) return MISA_EINVAL;
    if (n < 0) return fail(s, MISA_EINVAL, "step: n < 0");
    if (n == 0) return MISA_OK;
    s->energy_valid = false;
    s->ra_index_valid = false;
    if (s->use_graph && !s->timing) {
        int rc = s->prec == MISA_FP64 ? step_graph<double>(s, n, energy_last) : step_graph<float>(s, n, energy_last);
        if (rc) return rc;
    } else {
        for (int k = 0; k < n; ++k) {
            const bool e = energy_last && k == n - 1;
            int rc = s->prec == MISA_FP64 ? launch_step<double>(s, e) : launch_step<float>(s, e);
            if (rc) return rc;
        }
    }
    s->energy_valid = energy_last;
    s->ra_index_valid = false;
    return MISA_OK;
}

int misa_step(misa_sim *s, int n) { return step_impl(s, n, false); }

int misa_step_energies(misa_sim *s, int n)
{
    if (s && n < 1) return fail(s, MISA_EINVAL, "step_energies: n < 1");
    return step_impl(s, n, true);
}

int misa_set_species(misa_sim *s, int n_species, const double *f_knots, const double *F_knots,
                     const double *phi_knots, const int8_t *types)
{
    if (s) s->energy_valid = false;
    if (!s || n_species < 1 || n_species > kMaxSpecies || !f_knots || !F_knots || !phi_knots ||
        (n_species > 1 && !types))
        return s ? fail(s, MISA_EINVAL, "misa_set_species arguments") : MISA_EINVAL;
    int rc = s->prec == MISA_FP64 ? set_species_impl<double>(s, n_species, f_knots, F_knots, phi_knots, types)
                                  : set_species_impl<float>(s, n_species, f_knots, F_knots, phi_knots, types);
    return rc;
}

int misa_defects(misa_sim *s, int64_t *n_frenkel)
{
    if (!s || !n_frenkel) return MISA_EINVAL;
    unsigned long long *filled = reinterpret_cast<unsigned long long *>(s->partial);
    CK(cudaMemsetAsync(filled, 0, sizeof(unsigned long long) * s->nrep, s->st));
    if (s->prec == MISA_FP64) {
        k_defects_reset<double><<<list_grid(s), 256, 0, s->st>>>(md_args<double>(s), s->aux_int);
        k_defects_count<double><<<list_grid(s), 256, 0, s->st>>>(md_args<double>(s), s->aux_int, filled);
    } else {
        k_defects_reset<float><<<list_grid(s), 256, 0, s->st>>>(md_args<float>(s), s->aux_int);
        k_defects_count<float><<<list_grid(s), 256, 0, s->st>>>(md_args<float>(s), s->aux_int, filled);
    }
    CK(cudaGetLastError());
    std::vector<unsigned long long> f(s->nrep);
    std::vector<DevScalars> h(s->nrep);
    CK(cudaMemcpyAsync(f.data(), filled, sizeof(unsigned long long) * s->nrep, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(h.data(), s->sc, sizeof(DevScalars) * s->nrep, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    for (int r = 0; r < s->nrep; ++r) n_frenkel[r] = (int64_t)h[r].n_ra - (int64_t)f[r];
    s->launches += 2;
    return check_status(s);
}

int misa_retune(misa_sim *s)
{
    if (!s) return MISA_EINVAL;
    if (s->p.tile != 0) return MISA_OK;
    int rc = s->prec == MISA_FP64 ? autotune<double>(s) : autotune<float>(s);
    if (rc) return rc;
    return check_status(s);
}

int misa_set_density_variant(misa_sim *s, int32_t variant)
{
    if (s) s->energy_valid = false;
    if (!s) return MISA_EINVAL;
    if (variant != 0 && variant != 1)
        return fail(s, MISA_EINVAL, "density variant: 0 (full neighbour) or 1 (Newton's third law inside tiles)");
    if (variant == 1 && (s->prec != MISA_FP32_FORCE || s->nsp > 1))
        return fail(s, MISA_EINVAL, "the Newton-3 density pass is built for single-type FP32 handles");
    if (s->prec != MISA_FP32_FORCE || s->dens_n3 == (variant == 1)) return MISA_OK;
    const bool old = s->dens_n3;
    s->dens_n3 = variant == 1;
    int td = s->tile;
    if (!shape_fits<float>(s, td)) {
        td = 0;
        while (td < kNTiles && (!tile_ok(s->prec, kTiles[td]) || !shape_fits<float>(s, td))) ++td;
        if (td == kNTiles) {
            s->dens_n3 = old;
            return fail(s, MISA_EINVAL, "no tile shape fits the Newton-3 density pass's shared memory");
        }
    }
    int rc = configure<float>(s, td, s->tile_f);
    if (rc) {
        s->dens_n3 = old;
        configure<float>(s, s->tile, s->tile_f);
        return rc;
    }
    rc = refresh<float>(s, true);  // the current positions' forces through the new pass
    if (rc) return rc;
    return check_status(s);
}

int misa_set_graphs(misa_sim *s, int enable)
{
    if (!s) return MISA_EINVAL;
    s->use_graph = enable != 0;
    return MISA_OK;
}

int misa_get_energies_async(misa_sim *s, double *per_atom, int64_t n)
{
    if (!s) return MISA_EINVAL;
    if (!per_atom || n < s->ns) return fail(s, MISA_EINVAL, "get_energies_async: per_atom of natoms required");
    return s->prec == MISA_FP64 ? energies_async<double>(s, per_atom) : energies_async<float>(s, per_atom);
}

int misa_wait_outputs(misa_sim *s)
{
    if (!s) return MISA_EINVAL;
    if (s->ost) CK(cudaStreamSynchronize(s->ost));
    return check_status(s);
}

int misa_get_energies(misa_sim *s, double *pe, double *ke, double *per_atom)
{
    if (!s) return MISA_EINVAL;
    std::vector<double> p(s->nrep), k(s->nrep);
    int rc = s->prec == MISA_FP64 ? reduce_energy<double>(s, p.data(), k.data(), per_atom)
                                  : reduce_energy<float>(s, p.data(), k.data(), per_atom);
    if (rc) return rc;
    double P = 0.0, K = 0.0;
    for (int r = 0; r < s->nrep; ++r) {
        P += p[r];
        K += k[r];
    }
    if (pe) *pe = P;
    if (ke) *ke = K;
    return check_status(s);
}

int misa_replica_energies(misa_sim *s, double *pe, double *ke)
{
    if (!s) return MISA_EINVAL;
    int rc = s->prec == MISA_FP64 ? reduce_energy<double>(s, pe, ke, nullptr) : reduce_energy<float>(s, pe, ke, nullptr);
    if (rc) return rc;
    return check_status(s);
}

static int get_kind(misa_sim *s, int kind, double *out, int64_t n)
{
    if (!s) return MISA_EINVAL;
    if (!out || n < s->ns) return fail(s, MISA_EINVAL, "output buffer smaller than natoms");
    int rc = s->prec == MISA_FP64 ? scatter_out<double>(s, kind, out) : scatter_out<float>(s, kind, out);
    if (rc) return rc;
    return check_status(s);
}

int misa_get_positions(misa_sim *s, double *x, int64_t n) { return get_kind(s, 0, x, n); }
int misa_get_velocities(misa_sim *s, double *v, int64_t n) { return get_kind(s, 1, v, n); }
int misa_get_forces(misa_sim *s, double *f, int64_t n) { return get_kind(s, 2, f, n); }
int misa_get_density(misa_sim *s, double *rho, int64_t n) { return get_kind(s, 3, rho, n); }

int misa_get_site_map(misa_sim *s, int64_t *site_atom, int64_t *ra_ids, int64_t cap, int64_t *n_runaway)
{
    if (!s) return MISA_EINVAL;
    std::vector<DevScalars> h(s->nrep);
    CK(cudaMemcpyAsync(h.data(), s->sc, sizeof(DevScalars) * s->nrep, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    long long tot = 0;
    for (auto &q : h) tot += q.n_ra;
    if (n_runaway) *n_runaway = tot;
    if (ra_ids && cap < tot) return fail(s, MISA_EINVAL, "runaway_ids capacity too small");
    long long *d_sa = (long long *)s->aux_dbl;  // ns int64 fit in 3 ns doubles
    long long *d_ra = (long long *)s->out_buf;  // pooled run-away slots fit too
    if (s->prec == MISA_FP64) k_site_map<double><<<site_grid(s), 256, 0, s->st>>>(md_args<double>(s), d_sa, d_ra);
    else k_site_map<float><<<site_grid(s), 256, 0, s->st>>>(md_args<float>(s), d_sa, d_ra);
    if (site_atom) CK(cudaMemcpyAsync(site_atom, d_sa, sizeof(long long) * s->ns, cudaMemcpyDefault, s->st));
    if (ra_ids) {
        long long off = 0;
        for (int r = 0; r < s->nrep; ++r) {
            if (h[r].n_ra > 0)
                CK(cudaMemcpyAsync(ra_ids + off, d_ra + s->reps[r].ra_base, sizeof(long long) * h[r].n_ra,
                                   cudaMemcpyDefault, s->st));
            off += h[r].n_ra;
        }
    }
    CK(cudaStreamSynchronize(s->st));
    return MISA_OK;
}

int misa_stats_get(misa_sim *s, misa_stats *o)
{
    if (!s || !o) return MISA_EINVAL;
    std::vector<DevScalars> h(s->nrep);
    CK(cudaMemcpyAsync(h.data(), s->sc, sizeof(DevScalars) * s->nrep, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    DevScalars agg = h[0];
    agg.n_ra = 0;
    unsigned long long vb = 0;
    for (auto &q : h) {
        agg.n_ra += q.n_ra;
        vb = q.vmax_bits > vb ? q.vmax_bits : vb;
    }
    agg.vmax_bits = vb;
    stats_of(s, -1, agg, h[0].status, o);
    if (s->nrep > 1) o->dt = 0.0;  // replicas step with their own dt
    return MISA_OK;
}

int misa_replica_stats(misa_sim *s, int32_t r, misa_stats *o)
{
    if (!s || !o || r < 0 || r >= s->nrep) return MISA_EINVAL;
    std::vector<DevScalars> h(s->nrep);
    CK(cudaMemcpyAsync(h.data(), s->sc, sizeof(DevScalars) * s->nrep, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    return stats_of(s, r, h[r], h[0].status, o);
}

// 8 events per step: [start, after kick/drift, after list, after density,
// after ra density, after force, after ra force, after end]
int misa_timing_enable(misa_sim *s, int enable)
{
    if (!s) return MISA_EINVAL;
    CK(cudaStreamSynchronize(s->st));
    s->timing = enable != 0;
    s->ev_used = 0;
    return MISA_OK;
}

int misa_timing_get(misa_sim *s, double ms[MISA_NPHASE], int64_t *steps)
{
    if (!s || !ms) return MISA_EINVAL;
    CK(cudaStreamSynchronize(s->st));
    for (int k = 0; k < MISA_NPHASE; ++k) ms[k] = 0.0;
    const size_t per = MISA_NPHASE + 1;
    size_t nsteps = s->ev_used / per;
    for (size_t q = 0; q < nsteps; ++q)
        for (int k = 0; k < MISA_NPHASE; ++k) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, s->ev_pool[q * per + k], s->ev_pool[q * per + k + 1]));
            ms[k] += t;
        }
    if (steps) *steps = (int64_t)nsteps;
    s->ev_used = 0;
    return MISA_OK;
}

int misa_clear_status(misa_sim *s)
{
    if (!s) return MISA_EINVAL;
    CK(cudaMemsetAsync(&s->sc[0].status, 0, sizeof(unsigned), s->st));
    return MISA_OK;
}

// checkpoint: header, then the raw device arrays of the lattice list
struct CkptHeader {
    char magic[8];
    int32_t version, nrep, prec, cap;
    int64_t ns;
};

static int ckpt_io(misa_sim *s, const char *path, bool save)
{
    if (!s || !path) return MISA_EINVAL;
    CK(cudaStreamSynchronize(s->st));
    FILE *f = std::fopen(path, save ? "wb" : "rb");
    if (!f) return fail(s, MISA_EINVAL, std::string("cannot open ") + path);
    CkptHeader hd{};
    std::memcpy(hd.magic, "MISAGB3", 8);
    hd.version = 2; hd.nrep = s->nrep; hd.prec = s->prec; hd.cap = s->cap; hd.ns = s->ns;
    if (save) {
        std::fwrite(&hd, sizeof(hd), 1, f);
        std::fwrite(s->dims.data(), sizeof(int), s->dims.size(), f);
    } else {
        CkptHeader in{};
        std::vector<int> dims(s->dims.size());
        if (std::fread(&in, sizeof(in), 1, f) != 1 || std::memcmp(in.magic, hd.magic, 8) != 0 || in.version != 2 ||
            in.nrep != hd.nrep || in.prec != hd.prec || in.cap != hd.cap || in.ns != hd.ns ||
            std::fread(dims.data(), sizeof(int), dims.size(), f) != dims.size() || dims != s->dims) {
            std::fclose(f);
            return fail(s, MISA_EINVAL, "checkpoint does not match this handle");
        }
    }
    size_t Tb = s->prec == MISA_FP64 ? 8 : 4;
    const size_t capt = (size_t)s->cap * s->nrep;
    std::vector<std::pair<void *, size_t>> arrs = {{s->sid, 4 * (size_t)s->ns}, {s->sc, sizeof(DevScalars) * s->nrep}};
    for (int d = 0; d < 3; ++d) {
        arrs.push_back({s->u[d], 8 * (size_t)s->ns});
        arrs.push_back({s->v[d], 8 * (size_t)s->ns});
        arrs.push_back({s->a[d], Tb * (size_t)s->ns});
        if (s->prec != MISA_FP64) arrs.push_back({s->s[d], Tb * (size_t)s->ns});
        arrs.push_back({s->ra_u[d], 8 * capt});
        arrs.push_back({s->ra_v[d], 8 * capt});
        arrs.push_back({s->ra_s[d], Tb * capt});
        arrs.push_back({s->ra_a[d], Tb * capt});
    }
    arrs.push_back({s->ra_home, 4 * capt});
    arrs.push_back({s->ra_id, 4 * capt});
    std::vector<char> buf;
    int rc = MISA_OK;
    for (auto &a : arrs) {
        buf.resize(a.second);
        if (save) {
            if (cudaMemcpyAsync(buf.data(), a.first, a.second, cudaMemcpyDeviceToHost, s->st) != cudaSuccess ||
                cudaStreamSynchronize(s->st) != cudaSuccess) { rc = MISA_ECUDA; break; }
            if (std::fwrite(buf.data(), 1, a.second, f) != a.second) { rc = MISA_EINVAL; break; }
        } else {
            if (std::fread(buf.data(), 1, a.second, f) != a.second) { rc = MISA_EINVAL; break; }
            if (cudaMemcpyAsync(a.first, buf.data(), a.second, cudaMemcpyHostToDevice, s->st) != cudaSuccess ||
                cudaStreamSynchronize(s->st) != cudaSuccess) { rc = MISA_ECUDA; break; }
        }
    }
    std::fclose(f);
    if (rc) return fail(s, rc, "checkpoint i/o failed");
    return MISA_OK;
}

int misa_save(misa_sim *s, const char *path)
{
    if (s && s->nsp > 1) return fail(s, MISA_EINVAL, "checkpoints hold one atom type");
    return ckpt_io(s, path, true);
}
int misa_load(misa_sim *s, const char *path)
{
    if (s) s->energy_valid = s->ra_index_valid = false;
    return ckpt_io(s, path, false);
}

int misa_set_tables(misa_sim *s, const double *f_knots, const double *phi_knots, const double *F_knots)
{
    if (s) s->energy_valid = false;
    if (!s) return MISA_EINVAL;
    if (!f_knots || !phi_knots || !F_knots) return fail(s, MISA_EINVAL, "set_tables: three knot arrays required");
    return s->prec == MISA_FP64 ? set_tables_impl<double>(s, f_knots, phi_knots, F_knots)
                                : set_tables_impl<float>(s, f_knots, phi_knots, F_knots);
}

int misa_loss_grad(misa_sim *s, const double *Fref, const double *Eref, double *loss, double *grad)
{
    if (!s) return MISA_EINVAL;
    if (!Fref || !Eref) return fail(s, MISA_EINVAL, "loss_grad: targets required");
    int rc = s->prec == MISA_FP64 ? loss_grad_impl<double>(s, Fref, Eref, loss, grad)
                                  : loss_grad_impl<float>(s, Fref, Eref, loss, grad);
    if (rc) return rc;
    return check_status(s);
}

int misa_tile_count(void) { return kNTiles; }

int misa_tile_shape(int index, int *tx, int *ty, int *tz)
{
    if (index < 1 || index > kNTiles) return MISA_EINVAL;
    const TileShape &t = kTiles[index - 1];
    if (tx) *tx = t.tx;
    if (ty) *ty = t.ty;
    if (tz) *tz = t.tz;
    return MISA_OK;
}

int misa_tile_current(const misa_sim *s) { return s ? s->tile + 1 : 0; }

int misa_tile_current_force(const misa_sim *s) { return s ? s->tile_f + 1 : 0; }

int misa_selftest(long long n, long long *mismatches)
{
    if (n <= 0 || !mismatches) return MISA_EINVAL;
    unsigned long long *d = nullptr;
    unsigned long long h[3] = {0, 0, 0};
    if (cudaMalloc(&d, sizeof(h)) != cudaSuccess) return MISA_ECUDA;
    cudaError_t e = cudaMemset(d, 0, sizeof(h));
    if (e == cudaSuccess) {
        k_selftest_conv<<<1024, 256>>>((unsigned long long)n, d);
        k_selftest_site<<<1024, 256>>>((unsigned long long)n, d + 2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return MISA_ECUDA;
    mismatches[0] = (long long)h[0];
    mismatches[1] = (long long)h[1];
    mismatches[2] = (long long)h[2];
    return MISA_OK;
}

int misa_tile_valid(int precision, int index)
{
    if (index < 1 || index > kNTiles) return 0;
    if (precision != MISA_FP64 && precision != MISA_FP32_FORCE) return 0;
    return tile_ok(precision, kTiles[index - 1]) ? 1 : 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free force evaluation (misa_eam_forces_static)
// ---------------------------------------------------------------------------
// For callers that must not allocate device memory: all working memory of
// one force evaluation comes from this file-scope array.  Host code cannot
// use the symbol's host-side name as a device address; its device address is
// looked up once per device with cudaGetSymbolAddress.

namespace {

constexpr size_t kStaticAlign = 256;
// upper bound of the carve below for either precision: per site <= 160 B,
// per run-away slot <= 512 B, per knot <= 160 B, two flags and two map
// entries per cell (density and force tile maps), the two maps' run-away
// index (four ints per cell, 64 entries per run-away slot), two replica
// tables, the scalars, and the alignment padding
constexpr size_t kStaticNeed = 160ull * MISA_STATIC_MAX_ATOMS + 512ull * MISA_STATIC_RUNAWAY_CAP +
                               160ull * MISA_STATIC_MAX_KNOTS + 16ull * (MISA_STATIC_MAX_ATOMS / 2) +
                               2 * (16ull * (MISA_STATIC_MAX_ATOMS / 2) + 8 + 4 * 64ull * MISA_STATIC_RUNAWAY_CAP) +
                               sizeof(DevScalars) + 2 * sizeof(RepDesc) + 128 * kStaticAlign;
static_assert(kStaticNeed <= MISA_STATIC_SCRATCH_BYTES, "static scratch too small");

}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[MISA_STATIC_SCRATCH_BYTES];

namespace {

std::mutex g_static_mu;
void *g_static_addr[256] = {};  // device address of g_static_scratch, per device ordinal

struct Carver {
    unsigned char *base;
    size_t off = 0;
    template <typename X>
    X *take(size_t n)
    {
        off = (off + kStaticAlign - 1) & ~(kStaticAlign - 1);
        X *p = reinterpret_cast<X *>(base + off);
        off += sizeof(X) * n;
        return p;
    }
};

// Points every buffer of s into the static array; returns the bytes used.
template <typename T>
size_t carve_static(misa_sim *s, unsigned char *base, int nk)
{
    Carver c{base};
    const size_t ns = (size_t)s->ns, cap = (size_t)s->cap;
    s->reps_d = c.take<RepDesc>(1);
    s->sc = c.take<DevScalars>(1);
    s->sid = c.take<int>(ns);
    s->claim = c.take<int>(ns);
    for (int d = 0; d < 3; ++d) {
        s->u[d] = c.take<double>(ns);
        s->v[d] = c.take<double>(ns);
        s->a[d] = c.take<T>(ns);
        s->s[d] = sizeof(T) == 8 ? (void *)s->u[d] : (void *)c.take<T>(ns);
        s->ra_u[d] = c.take<double>(cap);
        s->ra_v[d] = c.take<double>(cap);
        s->ra_s[d] = c.take<T>(cap);
        s->ra_a[d] = c.take<T>(cap);
        s->t_u[d] = c.take<double>(cap);
        s->t_v[d] = c.take<double>(cap);
        s->t_s[d] = c.take<T>(cap);
        s->t_a[d] = c.take<T>(cap);
    }
    s->fp = c.take<T>(ns);
    s->rho = c.take<T>(ns);
    s->esite = c.take<double>(ns);
    if (sizeof(T) == 4) s->bmask = c.take<unsigned long long>(ns);
    s->ra_home = c.take<int>(cap);
    s->ra_id = c.take<int>(cap);
    s->t_home = c.take<int>(cap);
    s->t_id = c.take<int>(cap);
    s->ra_fp = c.take<T>(cap);
    s->ra_rho = c.take<T>(cap);
    s->ra_e = c.take<double>(cap);
    s->tab_f = c.take<Vec4<T>>(nk);
    s->tab_phi = c.take<Vec4<T>>(nk);
    s->tab_F = c.take<Vec4<T>>(nk);
    s->tab_d0 = c.take<Vec4<T>>(nk);
    s->tab_d1 = c.take<Vec2<T>>(nk);
    s->out_buf = c.take<double>(3 * ns);
    s->aux_int = c.take<int>(ns);
    s->tile_flag = c.take<int>(ns / 2);
    s->tile_rep = c.take<int>(ns / 2);
    s->reps_fd = c.take<RepDesc>(1);
    s->tile_flag_f = c.take<int>(ns / 2);
    s->tile_rep_f = c.take<int>(ns / 2);
    s->rt_cap = 64LL * (long long)cap;
    int *cnt2 = c.take<int>(ns);  // ntile_cap = ns / 2 per map
    int *aux2 = c.take<int>(4);
    for (int k = 0; k < 2; ++k) {
        s->rt_cnt[k] = cnt2 + (size_t)k * (ns / 2);
        s->rt_aux[k] = aux2 + 2 * k;
        s->rt_off[k] = c.take<int>(ns / 2);
        s->rt_fill[k] = c.take<int>(ns / 2);
        s->rt_nz[k] = c.take<int>(ns / 2);
        s->rt_list[k] = c.take<int>((size_t)s->rt_cap);
    }
    return c.off;
}

template <typename T>
int static_forces_impl(misa_sim *s, const double *knots, const double *x, double *forces, double *energies)
{
    const int n = s->p.n_knots;
    const double hr = s->p.rc / (n - 1), hrho = s->p.rho_max / (n - 1);
    // the scalars (step, time, list counts, status) start from zero on every call
    CK(cudaMemsetAsync(s->sc, 0, sizeof(DevScalars), s->st));
    k_spline_tables<T><<<(n + 255) / 256, 256, 0, s->st>>>(knots, knots + n, knots + 2 * n, n, hr, hrho,
                                                            (Vec4<T> *)s->tab_f, (Vec4<T> *)s->tab_phi,
                                                            (Vec4<T> *)s->tab_F, (Vec4<T> *)s->tab_d0,
                                                            (Vec2<T> *)s->tab_d1);
    int rc = configure<T>(s, 0, 0);
    if (rc) return rc;
    // hash the positions into the lattice list (clears sites, claims, list)
    // and evaluate forces; then the energy pass for E_i
    rc = set_state_impl<T>(s, x, nullptr);
    if (rc) return rc;
    MdArgs<T> m = md_args<T>(s);
    k_scatter<T><<<site_grid(s), 256, 0, s->st>>>(m, 2, s->out_buf);
    CK(cudaMemcpyAsync(forces, s->out_buf, sizeof(double) * 3 * (size_t)s->ns, cudaMemcpyDeviceToDevice, s->st));
    if (energies) {
        rc = launch_forces<T>(s, 0, true);
        if (rc) return rc;
        m = md_args<T>(s);
        k_scatter<T><<<site_grid(s), 256, 0, s->st>>>(m, 4, s->out_buf);
        CK(cudaMemcpyAsync(energies, s->out_buf, sizeof(double) * (size_t)s->ns, cudaMemcpyDeviceToDevice, s->st));
    }
    CK(cudaGetLastError());
    return check_status(s);
}

}  // namespace

extern "C" int misa_eam_forces_static(int32_t nx, int32_t ny, int32_t nz, double a0, double rc, double skin,
                                      int32_t n_knots, const double *knots, double rho_max, int32_t precision,
                                      const double *x, double *forces, double *energies, void *stream)
{
    misa_sim *none = nullptr;
    if (!knots || !x || !forces) return fail(none, MISA_EINVAL, "static forces: knots, x and forces are required");
    if (nx < 6 || ny < 6 || nz < 6) return fail(none, MISA_EINVAL, "static forces: each box dimension must be >= 6 cells");
    long long ns = 2LL * nx * ny * nz;
    if (ns > MISA_STATIC_MAX_ATOMS)
        return fail(none, MISA_EINVAL, "static forces: " + std::to_string(ns) + " atoms exceed the limit of " +
                                           std::to_string(MISA_STATIC_MAX_ATOMS));
    if (n_knots < 8 || n_knots > MISA_STATIC_MAX_KNOTS)
        return fail(none, MISA_EINVAL, "static forces: n_knots must be in [8, " + std::to_string(MISA_STATIC_MAX_KNOTS) + "]");
    if (!(a0 > 0) || !(rc > 0) || !(skin > 0) || !(rho_max > 0)) return fail(none, MISA_EINVAL, "static forces: a0, rc, skin, rho_max must be > 0");
    double half = 0.5 * a0, roff = (rc + 2.0 * skin) / half;
    if (roff * roff >= 27.0) return fail(none, MISA_EINVAL, "static forces: (rc + 2 skin) must be below sqrt(27) a0/2");
    if (skin >= 0.25 * std::sqrt(3.0) * a0) return fail(none, MISA_EINVAL, "static forces: skin too large");
    if (precision != MISA_FP64 && precision != MISA_FP32_FORCE) return fail(none, MISA_EINVAL, "static forces: precision");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256)
        return fail(none, MISA_ECUDA, "static forces: no current CUDA device");
    void *base = nullptr;
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess || !p)
                return fail(none, MISA_ECUDA, std::string("static forces: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_static_addr[dev] = p;
        }
        base = g_static_addr[dev];
    }

    misa_sim s;  // a handle on the host stack; every device buffer is carved from the static array
    misa_default_params(&s.p);
    s.p.nx = nx; s.p.ny = ny; s.p.nz = nz;
    s.p.a0 = a0; s.p.rc = rc; s.p.skin = skin;
    s.p.mass = 1.0;  // forces do not depend on it
    s.p.n_knots = n_knots;
    s.p.rho_max = rho_max;
    s.p.precision = precision;
    s.st = (cudaStream_t)stream;
    s.nrep = 1;
    s.ns = ns;
    s.prec = precision;
    s.cap = MISA_STATIC_RUNAWAY_CAP;
    s.reps.resize(1);
    std::memset(&s.reps[0], 0, sizeof(RepDesc));
    s.reps[0].nx = nx; s.reps[0].ny = ny; s.reps[0].nz = nz;
    s.reps[0].ns = ns;
    s.reps[0].cap = s.cap;
    s.ntile_cap = ns / 2;
    if (cudaDeviceGetAttribute(&s.nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || s.nsm <= 0)
        return fail(none, MISA_ECUDA, "static forces: cannot read the multiprocessor count of the device");
    size_t used = precision == MISA_FP64 ? carve_static<double>(&s, (unsigned char *)base, n_knots)
                                         : carve_static<float>(&s, (unsigned char *)base, n_knots);
    if (used > MISA_STATIC_SCRATCH_BYTES) return fail(none, MISA_EINVAL, "static forces: scratch layout exceeds the array");
    int r = precision == MISA_FP64 ? static_forces_impl<double>(&s, knots, x, forces, energies)
                                   : static_forces_impl<float>(&s, knots, x, forces, energies);
    if (r != MISA_OK) g_create_error = s.err;
    return r;
}
