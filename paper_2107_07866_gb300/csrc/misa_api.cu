// misa_api.cu -- host runtime and C ABI (include/misa.h) of the GB300 EAM
// lattice-list MD library.  Owns device memory, builds the neighbour offset
// index for the chosen tile shape (Sec. 3) and launches the step kernels on
// the handle's stream.  No host fallback: every step of the path runs in the
// kernels of misa_kernels.cuh / misa_md.cuh.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "misa.h"
#include "misa_md.cuh"

using namespace misa;

namespace {

constexpr double kAccUnit = 9.6485332123310018e-3;  // 1 eV/(A amu) in A/fs^2 (CODATA 2018)
constexpr double kRfloor = 1e-4;                      // A

struct TileShape {
    int tx, ty, tz;
};
constexpr TileShape kTiles[] = {{8, 8, 8}, {8, 8, 4}, {8, 4, 4}, {16, 8, 4}};
constexpr int kNTiles = sizeof(kTiles) / sizeof(kTiles[0]);

std::string g_create_error;

}  // namespace

struct misa_sim {
    misa_params p{};
    std::vector<double> fk, pk, Fk;
    cudaStream_t st = nullptr;
    int nx = 0, ny = 0, nz = 0;
    long long ns = 0;
    int prec = MISA_FP32_FORCE;
    int cap = 0;
    int tile = 0;
    int nsm = 0;
    std::string err;
    std::vector<std::pair<void *, size_t>> allocs;
    // device buffers
    int *sid = nullptr, *claim = nullptr, *tile_flag = nullptr;
    double *u[3] = {}, *v[3] = {};
    void *s[3] = {};   // precision-T shadow of u (FP32 path) or alias of u
    void *a[3] = {};
    void *fp = nullptr, *rho = nullptr;
    double *esite = nullptr;
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
    int ntx = 0, nty = 0, ntz = 0, ntiles = 0;
    size_t smem_density = 0, smem_force = 0;
    long long launches = 0;
    // phase timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<cudaEvent_t> cur;  // events of the step being launched
    long long timed_steps = 0;
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

template <typename T>
MdArgs<T> md_args(misa_sim *s)
{
    MdArgs<T> m{};
    m.nx = s->nx; m.ny = s->ny; m.nz = s->nz;
    m.ns = s->ns;
    m.sid = s->sid;
    m.ux = s->u[0]; m.uy = s->u[1]; m.uz = s->u[2];
    m.sx = (T *)s->s[0]; m.sy = (T *)s->s[1]; m.sz = (T *)s->s[2];
    m.vx = s->v[0]; m.vy = s->v[1]; m.vz = s->v[2];
    m.ax = (T *)s->a[0]; m.ay = (T *)s->a[1]; m.az = (T *)s->a[2];
    m.fp = (T *)s->fp; m.rho = (T *)s->rho;
    m.esite = s->esite;
    m.claim = s->claim;
    m.cap = s->cap;
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
    m.ntx = s->ntx; m.nty = s->nty; m.ntz = s->ntz;
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

template <typename T>
void fill_gather(misa_sim *s, GatherArgs<T> &g)
{
    std::memset(&g, 0, sizeof(g));
    const TileShape &ts = kTiles[s->tile];
    g.nx = s->nx; g.ny = s->ny; g.nz = s->nz;
    g.ntx = s->ntx; g.nty = s->nty; g.ntz = s->ntz; g.ntiles = s->ntiles;
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
    g.tile_flag = s->tile_flag;
    g.sc = s->sc;
    g.acc_conv = kAccUnit / s->p.mass;
    g.kick = 1;
    // neighbour offset index for this tile shape (Sec. 3): per parity, the
    // shared-memory slot displacement of every lattice vector
    const int SX = ts.tx + 4, SY = ts.ty + 4, SZ = ts.tz + 4;
    const int PLANE = SX * SY * SZ;
    for (int par = 0; par < 2; ++par)
        for (int k = 0; k < kNVec; ++k) {
            const LVec &o = kLVec.v[k];
            int pp = par ^ (o.x & 1);
            int D = (pp - par) * PLANE + (cell_shift(par, o.z) * SY + cell_shift(par, o.y)) * SX + cell_shift(par, o.x);
            float fD;
            std::memcpy(&fD, &D, sizeof(int));
            g.off[par][k] = make_float4(fD, 2.0f * o.x, 2.0f * o.y, 2.0f * o.z);
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
}

template <typename T>
size_t smem_density_bytes(misa_sim *s)
{
    const TileShape &ts = kTiles[s->tile];
    return gather_smem_bytes<T>(sizeof(T) == 4 ? sizeof(Vec4<T>) * (size_t)(s->p.n_knots - 1) : 0, ts.tx, ts.ty, ts.tz);
}

template <typename T>
size_t smem_force_bytes(misa_sim *s)
{
    const TileShape &ts = kTiles[s->tile];
    return gather_smem_bytes<T>(sizeof(T) == 4 ? (sizeof(Vec4<T>) + sizeof(Vec2<T>)) * (size_t)(s->p.n_knots - 1) : 0,
                                ts.tx, ts.ty, ts.tz);
}

// one instantiation of the tile kernels per tile shape
template <typename T, int TX, int TY, int TZ>
struct TileKernels {
    static int attrs(misa_sim *s)
    {
        CK(cudaFuncSetAttribute(k_density<T, TX, TY, TZ, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem_density));
        CK(cudaFuncSetAttribute(k_density<T, TX, TY, TZ, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem_density));
        CK(cudaFuncSetAttribute(k_force<T, TX, TY, TZ, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem_force));
        CK(cudaFuncSetAttribute(k_force<T, TX, TY, TZ, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem_force));
        return MISA_OK;
    }
    static void density(misa_sim *s, const GatherArgs<T> &g, int grid, bool energy)
    {
        constexpr int nt = 2 * TX * TY * TZ;
        if (energy) k_density<T, TX, TY, TZ, true><<<grid, nt, s->smem_density, s->st>>>(g);
        else k_density<T, TX, TY, TZ, false><<<grid, nt, s->smem_density, s->st>>>(g);
    }
    static void force(misa_sim *s, const GatherArgs<T> &g, int grid, bool energy)
    {
        constexpr int nt = 2 * TX * TY * TZ;
        if (energy) k_force<T, TX, TY, TZ, true><<<grid, nt, s->smem_force, s->st>>>(g);
        else k_force<T, TX, TY, TZ, false><<<grid, nt, s->smem_force, s->st>>>(g);
    }
};

// kTiles order: {8,8,8}, {8,8,4}, {8,4,4}, {16,8,4}
#define MISA_TILE_DISPATCH(T, idx, CALL)                      \
    switch (idx) {                                            \
    case 0: TileKernels<T, 8, 8, 8>::CALL; break;             \
    case 1: TileKernels<T, 8, 8, 4>::CALL; break;             \
    case 2: TileKernels<T, 8, 4, 4>::CALL; break;             \
    default: TileKernels<T, 16, 8, 4>::CALL; break;           \
    }

template <typename T>
int configure(misa_sim *s)
{
    const TileShape &ts = kTiles[s->tile];
    s->ntx = (s->nx + ts.tx - 1) / ts.tx;
    s->nty = (s->ny + ts.ty - 1) / ts.ty;
    s->ntz = (s->nz + ts.tz - 1) / ts.tz;
    s->ntiles = s->ntx * s->nty * s->ntz;
    s->smem_density = smem_density_bytes<T>(s);
    s->smem_force = smem_force_bytes<T>(s);
    int arc = MISA_OK;
    MISA_TILE_DISPATCH(T, s->tile, attrs(s) == MISA_OK ? (void)0 : (void)(arc = MISA_ECUDA));
    if (arc) return fail(s, arc, s->err.empty() ? "tile kernel attributes" : s->err);
    CK(cudaFuncSetAttribute(k_ra_sort<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)(sizeof(unsigned long long) * kSortMax)));
    if (s->tile_flag == nullptr) {
        // sized for the smallest tile shape so that re-tuning never reallocates
        long long maxt = 0;
        for (int k = 0; k < kNTiles; ++k) {
            long long nt = (long long)((s->nx + kTiles[k].tx - 1) / kTiles[k].tx) * ((s->ny + kTiles[k].ty - 1) / kTiles[k].ty) *
                           ((s->nz + kTiles[k].tz - 1) / kTiles[k].tz);
            maxt = nt > maxt ? nt : maxt;
        }
        s->tile_flag = (int *)dalloc(s, sizeof(int) * (size_t)maxt);
        if (!s->tile_flag) return fail(s, MISA_EOOM, "tile flags");
    }
    return MISA_OK;
}

template <typename T>
int launch_forces(misa_sim *s, int kick, bool energy, bool step_marks = false)
{
    MdArgs<T> m = md_args<T>(s);
    GatherArgs<T> g;
    fill_gather<T>(s, g);
    g.kick = kick;
    const int grid = s->ntiles < s->nsm ? s->ntiles : s->nsm;
    CK(cudaMemsetAsync(s->tile_flag, 0, sizeof(int) * (size_t)s->ntiles, s->st));
    k_mark_tiles<T><<<64, 256, 0, s->st>>>(m);
    RaGatherArgs<T> ra;
    std::memset(&ra, 0, sizeof(ra));
    ra.g = g;
    ra.sid = s->sid;
    ra.ra_sx = (const T *)s->ra_s[0]; ra.ra_sy = (const T *)s->ra_s[1]; ra.ra_sz = (const T *)s->ra_s[2];
    ra.ra_fp = (T *)s->ra_fp; ra.ra_rho = (T *)s->ra_rho; ra.ra_e = s->ra_e;
    ra.ra_ax = (T *)s->ra_a[0]; ra.ra_ay = (T *)s->ra_a[1]; ra.ra_az = (T *)s->ra_a[2];
    ra.ra_vx = s->ra_v[0]; ra.ra_vy = s->ra_v[1]; ra.ra_vz = s->ra_v[2];
    ra.energy = energy ? 1 : 0;
    if (step_marks) mark(s);  // end of the list phase
    MISA_TILE_DISPATCH(T, s->tile, density(s, g, grid, energy));
    if (step_marks) mark(s);
    k_ra_gather<T, 0><<<128, 256, 0, s->st>>>(ra);
    if (step_marks) mark(s);
    MISA_TILE_DISPATCH(T, s->tile, force(s, g, grid, energy));
    if (step_marks) mark(s);
    k_ra_gather<T, 1><<<128, 256, 0, s->st>>>(ra);
    if (step_marks) mark(s);
    s->launches += 5;
    CK(cudaGetLastError());
    return MISA_OK;
}

template <typename T>
int launch_step(misa_sim *s)
{
    MdArgs<T> m = md_args<T>(s);
    const int gs = s->nsm * 8;
    mark(s);
    k_begin_step<T><<<1, 1, 0, s->st>>>(m);
    k_ra_kick_drift<T><<<64, 256, 0, s->st>>>(m);
    k_kick_drift<T><<<gs, 256, 0, s->st>>>(m);
    mark(s);
    k_reassign_claim<T><<<64, 256, 0, s->st>>>(m, 0);
    k_reassign_promote<T><<<64, 256, 0, s->st>>>(m, 0);
    k_ra_sort<T><<<1, 1024, sizeof(unsigned long long) * kSortMax, s->st>>>(m);
    s->launches += 6;
    int rc = launch_forces<T>(s, 1, false, true);
    if (rc) return rc;
    k_end_step<T><<<1, 1, 0, s->st>>>(m);
    mark(s);
    s->launches += 1;
    if (s->timing) s->timed_steps += 1;
    CK(cudaGetLastError());
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
    CK(cudaMemsetAsync(&s->sc->vmax_bits, 0, sizeof(unsigned long long), s->st));
    k_vmax<T><<<s->nsm * 4, 256, 0, s->st>>>(m);
    CK(cudaGetLastError());
    return MISA_OK;
}

template <typename T>
int create_impl(misa_sim *s)
{
    const long long ns = s->ns;
    const int n = s->p.n_knots;
    size_t Tb = sizeof(T);
    s->sid = (int *)dalloc(s, sizeof(int) * ns);
    s->claim = (int *)dalloc(s, sizeof(int) * ns);
    for (int d = 0; d < 3; ++d) {
        s->u[d] = (double *)dalloc(s, sizeof(double) * ns);
        s->v[d] = (double *)dalloc(s, sizeof(double) * ns);
        s->a[d] = dalloc(s, Tb * ns);
        s->s[d] = sizeof(T) == 8 ? (void *)s->u[d] : dalloc(s, Tb * ns);
        s->ra_u[d] = (double *)dalloc(s, sizeof(double) * s->cap);
        s->ra_v[d] = (double *)dalloc(s, sizeof(double) * s->cap);
        s->ra_s[d] = dalloc(s, Tb * s->cap);
        s->ra_a[d] = dalloc(s, Tb * s->cap);
        s->t_u[d] = (double *)dalloc(s, sizeof(double) * s->cap);
        s->t_v[d] = (double *)dalloc(s, sizeof(double) * s->cap);
        s->t_s[d] = dalloc(s, Tb * s->cap);
        s->t_a[d] = dalloc(s, Tb * s->cap);
        if (!s->u[d] || !s->v[d] || !s->a[d] || !s->s[d] || !s->ra_u[d] || !s->ra_v[d] || !s->ra_s[d] || !s->ra_a[d] ||
            !s->t_u[d] || !s->t_v[d] || !s->t_s[d] || !s->t_a[d])
            return fail(s, MISA_EOOM, "device allocation failed");
    }
    s->fp = dalloc(s, Tb * ns);
    s->rho = dalloc(s, Tb * ns);
    s->esite = (double *)dalloc(s, sizeof(double) * ns);
    s->ra_home = (int *)dalloc(s, sizeof(int) * s->cap);
    s->ra_id = (int *)dalloc(s, sizeof(int) * s->cap);
    s->t_home = (int *)dalloc(s, sizeof(int) * s->cap);
    s->t_id = (int *)dalloc(s, sizeof(int) * s->cap);
    s->ra_fp = dalloc(s, Tb * s->cap);
    s->ra_rho = dalloc(s, Tb * s->cap);
    s->ra_e = (double *)dalloc(s, sizeof(double) * s->cap);
    s->knots = (double *)dalloc(s, sizeof(double) * 3 * n);
    s->tab_f = dalloc(s, sizeof(Vec4<T>) * n);
    s->tab_phi = dalloc(s, sizeof(Vec4<T>) * n);
    s->tab_F = dalloc(s, sizeof(Vec4<T>) * n);
    s->tab_d0 = dalloc(s, sizeof(Vec4<T>) * n);
    s->tab_d1 = dalloc(s, sizeof(Vec2<T>) * n);
    s->sc = (DevScalars *)dalloc(s, sizeof(DevScalars));
    s->partial = (double *)dalloc(s, sizeof(double) * 1024);
    s->red_out = (double *)dalloc(s, sizeof(double) * 2);
    s->out_buf = (double *)dalloc(s, sizeof(double) * 3 * ns);
    s->aux_int = (int *)dalloc(s, sizeof(int) * ns);
    s->aux_dbl = (double *)dalloc(s, sizeof(double) * 3 * ns);
    if (!s->fp || !s->rho || !s->esite || !s->ra_home || !s->ra_id || !s->t_home || !s->t_id || !s->ra_fp || !s->ra_rho ||
        !s->ra_e || !s->knots || !s->tab_f || !s->tab_phi || !s->tab_F || !s->tab_d0 || !s->tab_d1 || !s->sc ||
        !s->partial || !s->red_out || !s->out_buf || !s->aux_int || !s->aux_dbl)
        return fail(s, MISA_EOOM, "device allocation failed");
    CK(cudaMemcpyAsync(s->knots, s->fk.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->knots + n, s->pk.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->knots + 2 * n, s->Fk.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s->st));
    const double hr = s->p.rc / (n - 1), hrho = s->p.rho_max / (n - 1);
    k_spline_tables<T><<<(n + 255) / 256, 256, 0, s->st>>>(s->knots, s->knots + n, s->knots + 2 * n, n, hr, hrho,
                                                            (Vec4<T> *)s->tab_f, (Vec4<T> *)s->tab_phi,
                                                            (Vec4<T> *)s->tab_F, (Vec4<T> *)s->tab_d0,
                                                            (Vec2<T> *)s->tab_d1);
    int rc = configure<T>(s);
    if (rc) return rc;
    MdArgs<T> m = md_args<T>(s);
    k_init_crystal<T><<<s->nsm * 8, 256, 0, s->st>>>(m);
    CK(cudaGetLastError());
    return refresh<T>(s, true);
}

template <typename T>
int set_state_impl(misa_sim *s, const double *x, const double *v)
{
    const long long N = s->ns;
    MdArgs<T> m = md_args<T>(s);
    CK(cudaMemcpyAsync(s->out_buf, x, sizeof(double) * 3 * N, cudaMemcpyDefault, s->st));
    const double *vd = nullptr;
    if (v) {
        CK(cudaMemcpyAsync(s->aux_dbl, v, sizeof(double) * 3 * N, cudaMemcpyDefault, s->st));
        vd = s->aux_dbl;
    }
    k_reset_list<T><<<1, 1, 0, s->st>>>(m);
    k_clear_sites<T><<<s->nsm * 8, 256, 0, s->st>>>(m);
    const double L[3] = {s->nx * s->p.a0, s->ny * s->p.a0, s->nz * s->p.a0};
    // each atom's displacement from its nearest site overwrites its position in place
    k_state_claim<T><<<s->nsm * 8, 256, 0, s->st>>>(m, s->out_buf, N, L[0], L[1], L[2], s->aux_int, s->out_buf);
    if (!v) {
        CK(cudaMemsetAsync(s->v[0], 0, sizeof(double) * N, s->st));
        CK(cudaMemsetAsync(s->v[1], 0, sizeof(double) * N, s->st));
        CK(cudaMemsetAsync(s->v[2], 0, sizeof(double) * N, s->st));
    }
    k_state_place<T><<<s->nsm * 8, 256, 0, s->st>>>(m, vd, N, s->aux_int, s->out_buf);
    k_ra_sort<T><<<1, 1024, sizeof(unsigned long long) * kSortMax, s->st>>>(m);
    CK(cudaGetLastError());
    return refresh<T>(s, true);
}

template <typename T>
int reduce_energy(misa_sim *s, double *pe, double *ke, double *per_atom)
{
    int rc = launch_forces<T>(s, 0, true);
    if (rc) return rc;
    MdArgs<T> m = md_args<T>(s);
    const int nb = 512;
    k_sum_stage1<T><<<nb, 256, 0, s->st>>>(m, 0, s->partial);
    k_sum_stage2<<<1, 1024, 0, s->st>>>(s->partial, nb, s->red_out);
    k_sum_stage1<T><<<nb, 256, 0, s->st>>>(m, 1, s->partial);
    k_sum_stage2<<<1, 1024, 0, s->st>>>(s->partial, nb, s->red_out + 1);
    if (per_atom) {
        k_scatter<T><<<s->nsm * 8, 256, 0, s->st>>>(m, 4, s->out_buf, s->nx * s->p.a0, s->ny * s->p.a0, s->nz * s->p.a0);
        CK(cudaMemcpyAsync(per_atom, s->out_buf, sizeof(double) * s->ns, cudaMemcpyDefault, s->st));
    }
    double h[2];
    CK(cudaMemcpyAsync(h, s->red_out, sizeof(h), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    if (pe) *pe = h[0];
    if (ke) *ke = 0.5 * s->p.mass * h[1] / kAccUnit;
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
    k_scatter<T><<<s->nsm * 8, 256, 0, s->st>>>(m, kind, s->out_buf, s->nx * s->p.a0, s->ny * s->p.a0, s->nz * s->p.a0);
    CK(cudaGetLastError());
    size_t cnt = kind >= 3 ? (size_t)s->ns : 3 * (size_t)s->ns;
    CK(cudaMemcpyAsync(out, s->out_buf, sizeof(double) * cnt, cudaMemcpyDefault, s->st));
    CK(cudaStreamSynchronize(s->st));
    return MISA_OK;
}

int check_status(misa_sim *s)
{
    unsigned st = 0;
    CK(cudaMemcpyAsync(&st, &s->sc->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    if (st & kStRunawayOverflow) return fail(s, MISA_ERUNAWAY_OVERFLOW, "run-away list overflow");
    if (st & kStNonfinite) return fail(s, MISA_EUNSTABLE, "non-finite force or velocity");
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

int misa_create(const misa_params *pp, void *stream, misa_sim **out)
{
    misa_sim *s = nullptr;
    if (!pp || !out) return fail(s, MISA_EINVAL, "null argument");
    *out = nullptr;
    const misa_params &p = *pp;
    if (p.nx < 6 || p.ny < 6 || p.nz < 6) return fail(s, MISA_EINVAL, "each box dimension must be >= 6 cells");
    if (!(p.a0 > 0) || !(p.mass > 0) || !(p.rc > 0) || !(p.skin > 0)) return fail(s, MISA_EINVAL, "a0, mass, rc, skin must be > 0");
    if (p.n_knots < 8 || !p.f_knots || !p.phi_knots || !p.F_knots || !(p.rho_max > 0))
        return fail(s, MISA_EINVAL, "three knot tables (n >= 8) and rho_max > 0 are required");
    double half = 0.5 * p.a0, roff = (p.rc + 2.0 * p.skin) / half;
    if (roff * roff >= 27.0) return fail(s, MISA_EINVAL, "(rc + 2 skin) must be below sqrt(27) a0/2 (2-cell halo)");
    if (p.skin >= 0.25 * std::sqrt(3.0) * p.a0) return fail(s, MISA_EINVAL, "skin must be below half the nearest-neighbour distance");
    if (p.precision != MISA_FP64 && p.precision != MISA_FP32_FORCE) return fail(s, MISA_EINVAL, "precision");
    if (!(p.dt_max > 0) || p.dx_max < 0) return fail(s, MISA_EINVAL, "dt_max > 0, dx_max >= 0");
    if (!!p.alloc != !!p.free) return fail(s, MISA_EINVAL, "alloc and free hooks come together");
    long long ns = 2LL * p.nx * p.ny * p.nz;
    if (ns >= (1LL << 31)) return fail(s, MISA_EINVAL, "too many atoms for 32-bit ids");
    if (p.tile < 0 || p.tile > kNTiles) return fail(s, MISA_EINVAL, "tile index");
    s = new misa_sim();
    s->p = p;
    s->fk.assign(p.f_knots, p.f_knots + p.n_knots);
    s->pk.assign(p.phi_knots, p.phi_knots + p.n_knots);
    s->Fk.assign(p.F_knots, p.F_knots + p.n_knots);
    s->p.f_knots = s->fk.data();
    s->p.phi_knots = s->pk.data();
    s->p.F_knots = s->Fk.data();
    s->st = (cudaStream_t)stream;
    s->nx = p.nx; s->ny = p.ny; s->nz = p.nz;
    s->ns = ns;
    s->prec = p.precision;
    long long cap = p.runaway_capacity > 0 ? p.runaway_capacity : (ns / 64 > 4096 ? ns / 64 : 4096);
    if (cap > kSortMax) cap = kSortMax;
    s->cap = (int)cap;
    s->tile = p.tile > 0 ? p.tile - 1 : 0;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (s->nsm <= 0) s->nsm = 1;
    int rc = s->prec == MISA_FP64 ? create_impl<double>(s) : create_impl<float>(s);
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

void misa_destroy(misa_sim *s)
{
    if (!s) return;
    cudaStreamSynchronize(s->st);
    for (auto e : s->ev_pool) cudaEventDestroy(e);
    for (auto &a : s->allocs) {
        if (s->p.free) s->p.free(a.first, a.second, s->p.alloc_ctx);
        else cudaFree(a.first);
    }
    delete s;
}

const char *misa_last_error(const misa_sim *s) { return s ? s->err.c_str() : g_create_error.c_str(); }

int misa_set_state(misa_sim *s, const double *x, const double *v, int64_t n)
{
    if (!s) return MISA_EINVAL;
    if (!x || n != s->ns) return fail(s, MISA_EINVAL, "set_state: x required, n must equal natoms");
    return s->prec == MISA_FP64 ? set_state_impl<double>(s, x, v) : set_state_impl<float>(s, x, v);
}

int misa_set_velocities(misa_sim *s, const double *v, int64_t n)
{
    if (!s) return MISA_EINVAL;
    if (!v || n != s->ns) return fail(s, MISA_EINVAL, "set_velocities: n must equal natoms");
    CK(cudaMemcpyAsync(s->aux_dbl, v, sizeof(double) * 3 * s->ns, cudaMemcpyDefault, s->st));
    if (s->prec == MISA_FP64) {
        k_set_velocities<double><<<s->nsm * 8, 256, 0, s->st>>>(md_args<double>(s), s->aux_dbl);
        return refresh<double>(s, false);
    }
    k_set_velocities<float><<<s->nsm * 8, 256, 0, s->st>>>(md_args<float>(s), s->aux_dbl);
    return refresh<float>(s, false);
}

int misa_insert_pka(misa_sim *s, int64_t atom, double energy, const double dir[3])
{
    if (!s) return MISA_EINVAL;
    if (!dir || !(energy >= 0)) return fail(s, MISA_EINVAL, "insert_pka: bad direction or energy");
    double nrm = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    if (!(nrm > 0)) return fail(s, MISA_EINVAL, "insert_pka: zero direction");
    if (atom < 0) atom = 2LL * (((long long)(s->nz / 2) * s->ny + s->ny / 2) * s->nx + s->nx / 2);
    if (atom >= s->ns) return fail(s, MISA_EINVAL, "insert_pka: atom id out of range");
    double speed = std::sqrt(2.0 * energy / s->p.mass * kAccUnit);
    double vx = speed * dir[0] / nrm, vy = speed * dir[1] / nrm, vz = speed * dir[2] / nrm;
    if (s->prec == MISA_FP64) {
        k_pka<double><<<s->nsm * 8, 256, 0, s->st>>>(md_args<double>(s), (int)atom, vx, vy, vz);
        return refresh<double>(s, false);
    }
    k_pka<float><<<s->nsm * 8, 256, 0, s->st>>>(md_args<float>(s), (int)atom, vx, vy, vz);
    return refresh<float>(s, false);
}

int misa_step(misa_sim *s, int n)
{
    if (!s) return MISA_EINVAL;
    if (n < 0) return fail(s, MISA_EINVAL, "step: n < 0");
    for (int k = 0; k < n; ++k) {
        int rc = s->prec == MISA_FP64 ? launch_step<double>(s) : launch_step<float>(s);
        if (rc) return rc;
    }
    return MISA_OK;
}

int misa_get_energies(misa_sim *s, double *pe, double *ke, double *per_atom)
{
    if (!s) return MISA_EINVAL;
    int rc = s->prec == MISA_FP64 ? reduce_energy<double>(s, pe, ke, per_atom) : reduce_energy<float>(s, pe, ke, per_atom);
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
    DevScalars h;
    CK(cudaMemcpyAsync(&h, s->sc, sizeof(h), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    if (n_runaway) *n_runaway = h.n_ra;
    if (ra_ids && cap < h.n_ra) return fail(s, MISA_EINVAL, "runaway_ids capacity too small");
    long long *d_sa = (long long *)s->aux_dbl;          // ns int64 fit in 3 ns doubles
    long long *d_ra = (long long *)s->out_buf;
    if (s->prec == MISA_FP64) k_site_map<double><<<s->nsm * 8, 256, 0, s->st>>>(md_args<double>(s), d_sa, d_ra);
    else k_site_map<float><<<s->nsm * 8, 256, 0, s->st>>>(md_args<float>(s), d_sa, d_ra);
    if (site_atom) CK(cudaMemcpyAsync(site_atom, d_sa, sizeof(long long) * s->ns, cudaMemcpyDefault, s->st));
    if (ra_ids && h.n_ra > 0) CK(cudaMemcpyAsync(ra_ids, d_ra, sizeof(long long) * h.n_ra, cudaMemcpyDefault, s->st));
    CK(cudaStreamSynchronize(s->st));
    return MISA_OK;
}

int misa_stats_get(misa_sim *s, misa_stats *o)
{
    if (!s || !o) return MISA_EINVAL;
    DevScalars h;
    CK(cudaMemcpyAsync(&h, s->sc, sizeof(h), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    o->step = h.step;
    o->time = h.t;
    double vmax;
    std::memcpy(&vmax, &h.vmax_bits, sizeof(double));
    o->vmax = vmax;
    double dt = s->p.dt_max;
    if (s->p.dx_max > 0 && vmax > 0) dt = std::fmin(s->p.dt_max, s->p.dx_max / vmax);
    o->dt = dt;
    o->natoms = s->ns;
    o->nsites = s->ns;
    o->n_runaway = h.n_ra;
    o->n_vacant = h.n_ra;
    o->status = h.status;
    o->launches = s->launches;
    return MISA_OK;
}

// 8 events per step: [start, after kick/drift, after list, after density,
// after ra density, after force, after ra force, after end]
int misa_timing_enable(misa_sim *s, int enable)
{
    if (!s) return MISA_EINVAL;
    CK(cudaStreamSynchronize(s->st));
    s->timing = enable != 0;
    s->ev_used = 0;
    s->timed_steps = 0;
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
    s->timed_steps = 0;
    return MISA_OK;
}

int misa_clear_status(misa_sim *s)
{
    if (!s) return MISA_EINVAL;
    CK(cudaMemsetAsync(&s->sc->status, 0, sizeof(unsigned), s->st));
    return MISA_OK;
}

// checkpoint: header, then the raw device arrays of the lattice list
struct CkptHeader {
    char magic[8];
    int32_t version, nx, ny, nz, prec, cap;
};

static int ckpt_io(misa_sim *s, const char *path, bool save)
{
    if (!s || !path) return MISA_EINVAL;
    FILE *f = std::fopen(path, save ? "wb" : "rb");
    if (!f) return fail(s, MISA_EINVAL, std::string("cannot open ") + path);
    CkptHeader hd{};
    std::memcpy(hd.magic, "MISAGB3", 8);
    hd.version = 1; hd.nx = s->nx; hd.ny = s->ny; hd.nz = s->nz; hd.prec = s->prec; hd.cap = s->cap;
    if (save) {
        std::fwrite(&hd, sizeof(hd), 1, f);
    } else {
        CkptHeader in{};
        if (std::fread(&in, sizeof(in), 1, f) != 1 || std::memcmp(in.magic, hd.magic, 8) != 0 || in.nx != hd.nx ||
            in.ny != hd.ny || in.nz != hd.nz || in.prec != hd.prec || in.cap != hd.cap) {
            std::fclose(f);
            return fail(s, MISA_EINVAL, "checkpoint does not match this handle");
        }
    }
    size_t Tb = s->prec == MISA_FP64 ? 8 : 4;
    std::vector<std::pair<void *, size_t>> arrs = {{s->sid, 4 * (size_t)s->ns}, {s->sc, sizeof(DevScalars)}};
    for (int d = 0; d < 3; ++d) {
        arrs.push_back({s->u[d], 8 * (size_t)s->ns});
        arrs.push_back({s->v[d], 8 * (size_t)s->ns});
        arrs.push_back({s->a[d], Tb * (size_t)s->ns});
        if (s->prec != MISA_FP64) arrs.push_back({s->s[d], Tb * (size_t)s->ns});
        arrs.push_back({s->ra_u[d], 8 * (size_t)s->cap});
        arrs.push_back({s->ra_v[d], 8 * (size_t)s->cap});
        arrs.push_back({s->ra_s[d], Tb * (size_t)s->cap});
        arrs.push_back({s->ra_a[d], Tb * (size_t)s->cap});
    }
    arrs.push_back({s->ra_home, 4 * (size_t)s->cap});
    arrs.push_back({s->ra_id, 4 * (size_t)s->cap});
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

int misa_save(misa_sim *s, const char *path) { return ckpt_io(s, path, true); }
int misa_load(misa_sim *s, const char *path) { return ckpt_io(s, path, false); }

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
// per run-away slot <= 512 B, per knot <= 160 B, one flag per cell, the
// scalars, and the alignment padding of every buffer
constexpr size_t kStaticNeed = 160ull * MISA_STATIC_MAX_ATOMS + 512ull * MISA_STATIC_RUNAWAY_CAP +
                               160ull * MISA_STATIC_MAX_KNOTS + 4ull * (MISA_STATIC_MAX_ATOMS / 2) +
                               sizeof(DevScalars) + 96 * kStaticAlign;
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
    s->sc = c.take<DevScalars>(1);
    s->out_buf = c.take<double>(3 * ns);
    s->aux_int = c.take<int>(ns);
    s->tile_flag = c.take<int>(ns / 2);
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
    int rc = configure<T>(s);
    if (rc) return rc;
    // hash the positions into the lattice list (clears sites, claims, list)
    // and evaluate forces; then the energy pass for E_i
    rc = set_state_impl<T>(s, x, nullptr);
    if (rc) return rc;
    MdArgs<T> m = md_args<T>(s);
    const double L[3] = {s->nx * s->p.a0, s->ny * s->p.a0, s->nz * s->p.a0};
    k_scatter<T><<<s->nsm * 8, 256, 0, s->st>>>(m, 2, s->out_buf, L[0], L[1], L[2]);
    CK(cudaMemcpyAsync(forces, s->out_buf, sizeof(double) * 3 * (size_t)s->ns, cudaMemcpyDeviceToDevice, s->st));
    if (energies) {
        rc = launch_forces<T>(s, 0, true);
        if (rc) return rc;
        m = md_args<T>(s);
        k_scatter<T><<<s->nsm * 8, 256, 0, s->st>>>(m, 4, s->out_buf, L[0], L[1], L[2]);
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
    s.nx = nx; s.ny = ny; s.nz = nz;
    s.ns = ns;
    s.prec = precision;
    s.cap = MISA_STATIC_RUNAWAY_CAP;
    s.tile = 0;
    cudaDeviceGetAttribute(&s.nsm, cudaDevAttrMultiProcessorCount, dev);
    if (s.nsm <= 0) s.nsm = 1;
    size_t used = precision == MISA_FP64 ? carve_static<double>(&s, (unsigned char *)base, n_knots)
                                         : carve_static<float>(&s, (unsigned char *)base, n_knots);
    if (used > MISA_STATIC_SCRATCH_BYTES) return fail(none, MISA_EINVAL, "static forces: scratch layout exceeds the array");
    int r = precision == MISA_FP64 ? static_forces_impl<double>(&s, knots, x, forces, energies)
                                   : static_forces_impl<float>(&s, knots, x, forces, energies);
    if (r != MISA_OK) g_create_error = s.err;
    return r;
}
