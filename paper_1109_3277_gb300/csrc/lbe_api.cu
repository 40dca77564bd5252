// Host side of liblbe: context, device memory, the per-step launch
// sequence (captured in CUDA graphs) and the C ABI of include/lbe.h.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <algorithm>
#include <vector>

#include "lbe_internal.cuh"

using namespace lbe;

struct lbe_ctx {
    lbe_lattice_desc d{};
    int device = 0;
    Lat L{};
    Pair pair{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // the fused kernel's box copies of f[0], f[1]:
    // [ψ from memory, ψ formed in the kernel][8-row, 4-row tiles][buffer]
    CUtensorMap tmap[2][2][2];
    bool tma = false;
    size_t esize = 4;
    void *f[2] = {nullptr, nullptr};
    int cur = 0;
    float *rho = nullptr, *psi = nullptr;
    uint8_t *type = nullptr;
    uint32_t *owner[2] = {nullptr, nullptr};
    int ocur = 0;
    double *mass_partials = nullptr, *mass_out = nullptr;
    // particles
    int np = 0, cap = 0;
    double *pbuf = nullptr;
    float4 *x32 = nullptr;
    double *ppart = nullptr;
    void *geo = nullptr;   // coverage geometry records (cap of them)
    Parts P{};
    Cells cells{};   // pair-force cell list (with the particles)
    size_t cells_bytes = 0;
    LinkList ll{nullptr, nullptr, 0};  // link nodes of the step (allocated with the first particles)
    // graphs keyed by (cur, ocur)
    cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
    int zc_tuned = 0;  // fused-kernel z chunk chosen by lbe_autotune (0: heuristic)
    int ty_tuned = 8;  // fused-kernel tile rows chosen by lbe_autotune
    int wait_limit = FUSED_WAIT_LIMIT;  // tries of each bounded wait for a box copy
    // profiling
    bool profiling = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    size_t bytes = 0;
    std::string err;
};

namespace {

lbe_status fail(lbe_ctx *c, lbe_status st, const std::string &m)
{
    if (c) c->err = m;
    return st;
}

lbe_status cuda_fail(lbe_ctx *c, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? LBE_ENOMEM : LBE_ECUDA, m);
}

#define CK(c, call)                                            \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
    } while (0)

size_t storage_size(int s) { return s == LBE_STORE_F32 ? 4 : 2; }

void drop_graphs(lbe_ctx *c)
{
    for (auto &g : c->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// Field offsets inside the particle buffer (doubles per particle).
enum { OX = 0, OQ = 3, OV = 7, OW = 10, OXO = 13, OQO = 16, ORP = 20, ORO = 21, ODR = 22, OM = 23,
       OIP = 24, OIQ = 25, OFL = 26, OTL = 29, OFP = 32, OTP = 35, OFE = 38, OTE = 41, OF = 44,
       OT = 47, OFX = 50, PSTRIDE = 56 };

void bind_parts(lbe_ctx *c)
{
    // structure of arrays: field k occupies [k*cap, (k+1)*cap) doubles
    double *b = c->pbuf;
    size_t cp = (size_t)c->cap;
    auto at = [&](int off) { return b + (size_t)off * cp; };
    Parts &P = c->P;
    P.n = c->np;
    P.X = at(OX);
    P.q = at(OQ);
    P.V = at(OV);
    P.W = at(OW);
    P.Xold = at(OXO);
    P.qold = at(OQO);
    P.rp = at(ORP);
    P.ro = at(ORO);
    P.drho = at(ODR);
    P.M = at(OM);
    P.Ipar = at(OIP);
    P.Iperp = at(OIQ);
    P.Flink = at(OFL);
    P.Tlink = at(OTL);
    P.Fpair = at(OFP);
    P.Tpair = at(OTP);
    P.Fpend = at(OFE);
    P.Tpend = at(OTE);
    P.F = at(OF);
    P.T = at(OT);
    P.fix = reinterpret_cast<unsigned long long *>(at(OFX));
    P.X32 = c->x32;
    P.K32 = c->x32 ? c->x32 + c->cap : nullptr;
    P.ppart = c->ppart;
    P.geo = c->geo;
    P.nsplit = 1;
}

void free_all(lbe_ctx *c)
{
    drop_graphs(c);
    for (auto &e : c->ev) cudaEventDestroy(e);
    c->ev.clear();
    cudaFree(c->f[0]);
    cudaFree(c->f[1]);
    cudaFree(c->rho);
    cudaFree(c->psi);
    cudaFree(c->type);
    cudaFree(c->owner[0]);
    cudaFree(c->owner[1]);
    cudaFree(c->mass_partials);
    cudaFree(c->mass_out);
    cudaFree(c->pbuf);
    cudaFree(c->x32);
    cudaFree(c->ppart);
    cudaFree(c->geo);
    cudaFree(c->cells.count);
    cudaFree(c->cells.idx);
    cudaFree(c->ll.ent);
    cudaFree(c->ll.count);
    if (c->L.err) cudaFree(c->L.err);
    cudaFree(c->L.status);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

// Allocation-failure injection (lbe_fail_allocations): the number of device
// allocations still allowed, or -1 for no limit.
std::atomic<int> g_alloc_left{-1};

bool alloc_refused()
{
    int n = g_alloc_left.load();
    while (n >= 0) {
        if (n == 0) return true;
        if (g_alloc_left.compare_exchange_weak(n, n - 1)) return false;
    }
    return false;
}

// Every device allocation of a context goes through these two.
cudaError_t lib_malloc(void **p, size_t bytes)
{
    if (alloc_refused()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t lib_malloc_async(void **p, size_t bytes, cudaStream_t s)
{
    if (alloc_refused()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(p, bytes, s);
}

template <class T>
cudaError_t dalloc(lbe_ctx *c, T **p, size_t bytes)
{
    cudaError_t e = lib_malloc((void **)p, bytes);
    if (e == cudaSuccess) c->bytes += bytes;
    return e;
}

__global__ void k_set_types(Lat L, uint8_t *type)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= L.N) return;
    int z = n / (L.nx * L.ny);
    type[n] = (L.walls && (z == 0 || z == L.nz - 1)) ? WALL : FLUID;
}

// The fused kernel forms ψ of the fluid nodes itself when no particle needs
// the densities from memory (a lattice without particles runs no density
// kernel); with particles, the density kernel feeds the shell fill and the
// fused kernel reads ψ.
bool fused_self(const lbe_ctx *c) { return c->np == 0; }

// Tensor map of buffer `buf` for the fused kernel's mode and tile height
// (null without TMA).
const CUtensorMap *fused_map(const lbe_ctx *c, int buf, int ty)
{
    if (!c->tma) return nullptr;
    return &c->tmap[fused_self(c) ? 1 : 0][fused_rows(c->L, ty, true) == 4 ? 1 : 0][buf];
}

// Enqueue one time step (no host synchronisation).
void enqueue_step(lbe_ctx *c)
{
    cudaStream_t s = c->stream;
    const Lat &L = c->L;
    int st = c->d.storage;
    void *fin = c->f[c->cur], *fout = c->f[1 - c->cur];
    const bool two_pass = (c->d.flags & LBE_FLAG_TWO_PASS) != 0;
    const bool links = c->np > 0 && !two_pass;
    if (two_pass) {
        launch_moments(st, L, fin, c->type, c->rho, c->psi, s);
        launch_shell(L, c->rho, c->psi, c->type, c->owner[c->ocur], c->P.drho, LinkList{nullptr, nullptr, 0}, s);
    } else {
        if (links) cudaMemsetAsync(c->ll.count, 0, sizeof(int), s);
        // the solid nodes a fluid node can see: the particles' own nodes and
        // the wall planes (none for a periodic lattice without particles);
        // without particles the fused kernel forms the densities itself
        if (c->np > 0) {
            c->P.n = c->np;
            launch_rho(st, L, fin, c->type, c->rho, c->psi, s);
            launch_shell_particles(L, c->P, c->rho, c->psi, c->type, c->owner[c->ocur], c->ll, s);
        }
        launch_shell_walls(st, L, fin, c->psi, c->type, s);
    }
    if (c->profiling) {
        if (c->ev_used + 2 > c->ev.size()) {
            for (int k = 0; k < 256; k++) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                c->ev.push_back(e);
            }
        }
        cudaEventRecord(c->ev[c->ev_used], s);
    }
    if (two_pass)
        launch_collide_stream(st, L, fin, fout, c->psi, c->type, s);
    else
        launch_fused(st, L, fin, fout, c->psi, c->type, fused_map(c, c->cur, c->ty_tuned), s, c->zc_tuned,
                     c->ty_tuned, c->wait_limit, fused_self(c));
    if (c->profiling) {
        cudaEventRecord(c->ev[c->ev_used + 1], s);
        c->ev_used += 2;
    }
    if (c->np > 0) {
        c->P.n = c->np;
        if (two_pass)
            launch_links(st, L, c->P, fout, c->rho, c->type, c->owner[c->ocur], s);
        else {
            launch_link(st, L, c->ll, c->rho, c->owner[c->ocur], c->P, fout, s);
            // the list is empty between steps (batched steps rely on it)
            cudaMemsetAsync(c->ll.count, 0, sizeof(int), s);
        }
        launch_pairs(L, c->P, c->pair, c->cells, s);
        launch_integrate(L, c->P, c->d.particle_mode, s);
        if (c->d.particle_mode != LBE_PARTICLES_STATIC) {
            uint32_t *oo = c->owner[c->ocur], *on = c->owner[1 - c->ocur];
            launch_geom(L, c->P, s);
            launch_claim(L, c->P, 0, on, s);
            launch_transition(st, L, c->P, fout, c->type, oo, on, 0, s);
            launch_reset(L, c->P, 1, oo, s);
            c->ocur = 1 - c->ocur;
            launch_verify(L, c->type, on, s);
        }
    }
    c->cur = 1 - c->cur;
}

// Cell list for the pair forces: cells of edge >= the largest pair reach
// (2 max radius + Δc + the prefilter's margin), at least 2 nodes a side.
// (np particles of the block blk laid out for capacity cap; on failure the
// context keeps its old cells)
lbe_status build_cells(lbe_ctx *c, const std::vector<double> &blk, int cap, int np)
{
    double rmax = 0.0;
    for (int p = 0; p < np; p++)
        rmax = std::fmax(rmax, std::fmax(blk[(size_t)ORP * cap + p], blk[(size_t)ORO * cap + p]));
    const double reach = 2.0 * rmax + c->pair.lub_cut + 0.1;
    Cells &C = c->cells;
    const int dim[3] = {c->L.nx, c->L.ny, c->L.nz};
    long long ncell = 1;
    int cn[3];
    float cinv[3];
    for (int k = 0; k < 3; k++) {
        int n = (int)std::floor(dim[k] / reach);
        n = std::max(1, std::min(n, dim[k] / 2));
        cn[k] = n;
        cinv[k] = (float)((double)n / dim[k]);
        ncell *= n;
    }
    // count | start | fill in one buffer, idx | cid in another; the old
    // buffers go only once the new ones exist
    const size_t b0 = (size_t)(3 * ncell + 1) * sizeof(int), b1 = (size_t)2 * cap * sizeof(int);
    int *ncount = nullptr, *nidx = nullptr;
    cudaError_t e = lib_malloc((void **)&ncount, b0);
    if (e != cudaSuccess) return cuda_fail(c, e, "add_particles: cudaMalloc(cells)");
    e = lib_malloc((void **)&nidx, b1);
    if (e != cudaSuccess) {
        cudaFree(ncount);
        return cuda_fail(c, e, "add_particles: cudaMalloc(cells)");
    }
    if (C.count) {
        cudaFree(C.count);
        cudaFree(C.idx);
        c->bytes -= c->cells_bytes;
    }
    C.count = ncount;
    C.idx = nidx;
    C.ncell = (int)ncell;
    for (int k = 0; k < 3; k++) {
        C.n[k] = cn[k];
        C.inv[k] = cinv[k];
    }
    C.start = C.count + ncell;
    C.fill = C.start + ncell + 1;
    C.cid = C.idx + cap;
    c->cells_bytes = b0 + b1;
    c->bytes += c->cells_bytes;
    return LBE_OK;
}

lbe_status check_async(lbe_ctx *c, const char *where)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, where);
    return LBE_OK;
}

lbe_status sync(lbe_ctx *c, const char *where)
{
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, where);
    unsigned status = 0;
    if (c->L.status && cudaMemcpy(&status, c->L.status, sizeof status, cudaMemcpyDeviceToHost) == cudaSuccess &&
        (status & 1u))
        return fail(c, LBE_ETIMEOUT, std::string(where) + ": a plane copy of the fused kernel did not complete");
#ifdef LBE_CHECK
    unsigned long long bad = 0;
    if (c->L.err && cudaMemcpy(&bad, c->L.err, sizeof bad, cudaMemcpyDeviceToHost) == cudaSuccess && bad) {
        char m[128];
        snprintf(m, sizeof m, "%s: bounds check failed: site %llu index %llu", where, bad >> 40,
                 bad & 0xFFFFFFFFFFull);
        return fail(c, LBE_ECUDA, m);
    }
#endif
    return check_async(c, where);
}

}  // namespace

extern "C" {

lbe_status lbe_init_lattice(const lbe_lattice_desc *d, const double *rho0, lbe_ctx **out)
{
    if (!d || !rho0 || !out) return LBE_EINVAL;
    *out = nullptr;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return LBE_EINVAL;
    if (d->walls_z && d->nz < 3) return LBE_EINVAL;
    if (!(d->tau[0] > 0.5) || !(d->tau[1] > 0.5)) return LBE_EINVAL;
    if (d->storage < LBE_STORE_F32 || d->storage > LBE_STORE_F16_OFS) return LBE_EINVAL;
    if (d->particle_mode < 0 || d->particle_mode > 2) return LBE_EINVAL;
    if (d->flags & ~(LBE_FLAG_TWO_PASS | LBE_FLAG_WIDE_OFFSETS)) return LBE_EINVAL;
    if (!(d->rho_particle >= 0) || !(d->rho_particle < 1e30)) return LBE_EINVAL;
    long long N = (long long)d->nx * d->ny * d->nz;
    if (N > 0x7fffffffLL) return LBE_EINVAL;
    if (d->ny > 65535 || d->nz > 65535) return LBE_EINVAL;  // launch-grid rows and planes
    int dev = d->device;
    if (dev >= 0) {
        if (cudaSetDevice(dev) != cudaSuccess) return LBE_EINVAL;
    } else if (cudaGetDevice(&dev) != cudaSuccess) {
        return LBE_ECUDA;
    }
    lbe_ctx *c = new (std::nothrow) lbe_ctx();
    if (!c) return LBE_ENOMEM;
    c->d = *d;
    c->device = dev;
    Lat &L = c->L;
    L.nx = d->nx;
    L.ny = d->ny;
    L.nz = d->nz;
    L.walls = d->walls_z ? 1 : 0;
    L.N = (int)N;
    L.S = ((N + 127) / 128) * 128 + 384;
    L.wide = (d->flags & LBE_FLAG_WIDE_OFFSETS) ? 1 : 0;
    for (int k = 0; k < 2; k++) {
        L.tau[k] = (float)d->tau[k];
        L.itau[k] = (float)(1.0 / d->tau[k]);
        L.rho_ref[k] = d->rho_ref[k];
        L.rref[k] = d->storage == LBE_STORE_F32 ? 0.f : (float)d->rho_ref[k];
        for (int i = 0; i < Q; i++)
            L.base[k][i] = d->storage == LBE_STORE_F32 ? 0.f : (float)(wgtd(i) * d->rho_ref[k]);
    }
    L.g = (float)d->g_br;
    for (int k = 0; k < 3; k++) L.body[k] = (float)d->body_force[k];
    c->pair.k_hertz = d->k_hertz;
    c->pair.lub_cut = d->lub_cut;
    c->pair.mu = d->lub_rho * ((0.5 * (d->tau[0] + d->tau[1]) - 0.5) / 3.0);
    c->pair.mode = d->particle_mode;
    c->esize = storage_size(d->storage);
    lbe_status st = LBE_OK;
    auto bail = [&](cudaError_t e, const char *w) {
        st = cuda_fail(c, e, w);
        free_all(c);
        delete c;
        return st;
    };
    cudaError_t e;
    if (d->cuda_stream) {
        c->stream = (cudaStream_t)d->cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(e, "cudaStreamCreate");
        c->own_stream = true;
    }
    size_t fbytes = (size_t)2 * Q * L.S * c->esize;
    if ((e = dalloc(c, &c->f[0], fbytes)) != cudaSuccess) return bail(e, "cudaMalloc(f0)");
    if ((e = dalloc(c, &c->f[1], fbytes)) != cudaSuccess) return bail(e, "cudaMalloc(f1)");
    if ((e = dalloc(c, &c->rho, (size_t)2 * N * sizeof(float))) != cudaSuccess) return bail(e, "cudaMalloc(rho)");
    if ((e = dalloc(c, &c->psi, (size_t)2 * N * sizeof(float))) != cudaSuccess) return bail(e, "cudaMalloc(psi)");
    if ((e = dalloc(c, &c->type, (size_t)N)) != cudaSuccess) return bail(e, "cudaMalloc(type)");
    if ((e = dalloc(c, &c->owner[0], (size_t)N * 4)) != cudaSuccess) return bail(e, "cudaMalloc(owner0)");
    if ((e = dalloc(c, &c->owner[1], (size_t)N * 4)) != cudaSuccess) return bail(e, "cudaMalloc(owner1)");
    if ((e = dalloc(c, &c->mass_partials, (size_t)2 * mass_blocks() * sizeof(double))) != cudaSuccess)
        return bail(e, "cudaMalloc(mass)");
    if ((e = dalloc(c, &c->mass_out, 2 * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc(mass_out)");
    if ((e = dalloc(c, &c->L.status, sizeof(unsigned))) != cudaSuccess) return bail(e, "cudaMalloc(status)");
    cudaMemsetAsync(c->L.status, 0, sizeof(unsigned), c->stream);
    c->tma = true;
    for (int m = 0; m < 2; m++)
        for (int t = 0; t < 2; t++)
            for (int b = 0; b < 2; b++)
                c->tma = c->tma && fused_plane_map(&c->tmap[m][t][b], c->f[b], L, d->storage, t == 0 ? 8 : 4, m == 1);
#ifdef LBE_CHECK
    if ((e = cudaMalloc((void **)&c->L.err, sizeof(unsigned long long))) != cudaSuccess) return bail(e, "cudaMalloc(err)");
    cudaMemset(c->L.err, 0, sizeof(unsigned long long));
#endif
    cudaStream_t s = c->stream;
    cudaMemsetAsync(c->owner[0], 0xFF, (size_t)N * 4, s);
    cudaMemsetAsync(c->owner[1], 0xFF, (size_t)N * 4, s);
    cudaMemsetAsync(c->rho, 0, (size_t)2 * N * sizeof(float), s);
    cudaMemsetAsync(c->psi, 0, (size_t)2 * N * sizeof(float), s);
    cudaMemsetAsync(c->f[1], 0, fbytes, s);
    k_set_types<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(L, c->type);
    double *drho0 = nullptr;
    if ((e = lib_malloc_async((void **)&drho0, (size_t)2 * N * sizeof(double), s)) != cudaSuccess)
        return bail(e, "cudaMallocAsync(rho0)");
    cudaMemcpyAsync(drho0, rho0, (size_t)2 * N * sizeof(double), cudaMemcpyHostToDevice, s);
    launch_init_f(d->storage, L, drho0, c->f[0], c->type, s);
    cudaFreeAsync(drho0, s);
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return bail(e, "init");
    bind_parts(c);
    *out = c;
    return LBE_OK;
}

lbe_status lbe_add_particles(lbe_ctx *c, int32_t n, const double *pos, const double *quat,
                             const double *vel, const double *omega, const double *r_par,
                             const double *r_perp, const double *delta_rho)
{
    if (!c) return LBE_EINVAL;
    cudaSetDevice(c->device);
    if (n < 0 || (n > 0 && (!pos || !quat || !r_par || !r_perp || !delta_rho)))
        return fail(c, LBE_EINVAL, "add_particles: bad arguments");
    if (n == 0) return LBE_OK;
    int ext[3] = {c->d.nx, c->d.ny, c->d.nz};
    for (int k = 0; k < n; k++) {
        if (!(r_par[k] > 0) || !(r_perp[k] > 0)) return fail(c, LBE_EINVAL, "add_particles: radii must be positive");
        double qq = quat[4 * k] * quat[4 * k] + quat[4 * k + 1] * quat[4 * k + 1] +
                    quat[4 * k + 2] * quat[4 * k + 2] + quat[4 * k + 3] * quat[4 * k + 3];
        if (!(qq > 0)) return fail(c, LBE_EINVAL, "add_particles: zero quaternion");
        for (int j = 0; j < 3; j++)
            if (!(pos[3 * k + j] >= 0) || !(pos[3 * k + j] < ext[j]))
                return fail(c, LBE_EINVAL, "add_particles: position outside the lattice");
    }
    lbe_status st = sync(c, "add_particles");
    if (st != LBE_OK) return st;
    static const int FIELDS[][2] = {{OX, 3},  {OQ, 4},  {OV, 3},  {OW, 3},  {OXO, 3}, {OQO, 4}, {ORP, 1},
                                    {ORO, 1}, {ODR, 1}, {OM, 1},  {OIP, 1}, {OIQ, 1}, {OFL, 3}, {OTL, 3},
                                    {OFP, 3}, {OTP, 3}, {OFE, 3}, {OTE, 3}, {OF, 3},  {OT, 3},
                                    {OFX, 6}};
    // Each field of width k occupies k*cap doubles starting at off*cap; the
    // live state of existing particles is read back and re-laid for the new
    // capacity.
    int old = c->np, cap = c->cap, np = old + n;
    int ncap = np > cap ? (np < 64 ? 64 : np + np / 4) : cap;
    std::vector<double> oldb;
    if (old > 0) {
        oldb.resize((size_t)PSTRIDE * cap);
        CK(c, cudaMemcpy(oldb.data(), c->pbuf, oldb.size() * sizeof(double), cudaMemcpyDeviceToHost));
    }
    std::vector<double> blk((size_t)PSTRIDE * ncap, 0.0);
    for (auto &fk : FIELDS)
        for (size_t e2 = 0; e2 < (size_t)fk[1] * old; e2++)
            blk[(size_t)fk[0] * ncap + e2] = oldb[(size_t)fk[0] * cap + e2];
    size_t cp = (size_t)ncap;
    for (int k = 0; k < n; k++) {
        int p = old + k;
        double qn = std::sqrt(((quat[4 * k] * quat[4 * k] + quat[4 * k + 1] * quat[4 * k + 1]) +
                               quat[4 * k + 2] * quat[4 * k + 2]) + quat[4 * k + 3] * quat[4 * k + 3]);
        for (int j = 0; j < 3; j++) {
            blk[OX * cp + 3 * p + j] = pos[3 * k + j];
            blk[OV * cp + 3 * p + j] = vel ? vel[3 * k + j] : 0.0;
            blk[OW * cp + 3 * p + j] = omega ? omega[3 * k + j] : 0.0;
        }
        for (int j = 0; j < 4; j++) blk[OQ * cp + 4 * p + j] = quat[4 * k + j] / qn;
        double rp = r_par[k], ro = r_perp[k];
        // mass density ρ_p of the descriptor (the paper gives none; 0 means
        // 1), solid-ellipsoid inertia
        const double rho_p = c->d.rho_particle > 0 ? c->d.rho_particle : 1.0;
        double M = rho_p * 4.0 / 3.0 * M_PI * rp * ro * ro;
        blk[ORP * cp + p] = rp;
        blk[ORO * cp + p] = ro;
        blk[ODR * cp + p] = delta_rho[k];
        blk[OM * cp + p] = M;
        blk[OIP * cp + p] = 0.4 * M * ro * ro;
        blk[OIQ * cp + p] = 0.2 * M * (rp * rp + ro * ro);
    }
    // placement does not move anything: old geometry = current geometry
    for (int p = 0; p < np; p++) {
        for (int j = 0; j < 3; j++) blk[OXO * cp + 3 * p + j] = blk[OX * cp + 3 * p + j];
        for (int j = 0; j < 4; j++) blk[OQO * cp + 4 * p + j] = blk[OQ * cp + 4 * p + j];
    }
    // FP32 copies: [0, ncap) position and reach, then velocity and ω pairs
    std::vector<float4> x32((size_t)3 * ncap, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int p = 0; p < np; p++) {
        x32[p] = make_float4((float)blk[OX * cp + 3 * p], (float)blk[OX * cp + 3 * p + 1],
                             (float)blk[OX * cp + 3 * p + 2], (float)std::fmax(blk[ORP * cp + p], blk[ORO * cp + p]));
        x32[ncap + 2 * p] = make_float4((float)blk[OV * cp + 3 * p], (float)blk[OV * cp + 3 * p + 1],
                                        (float)blk[OV * cp + 3 * p + 2], 0.f);
        x32[ncap + 2 * p + 1] = make_float4((float)blk[OW * cp + 3 * p], (float)blk[OW * cp + 3 * p + 1],
                                            (float)blk[OW * cp + 3 * p + 2], 0.f);
    }
    if (!c->ll.ent) {
        // a fluid node enters the link list at most once per step: N entries
        uint2 *ent = nullptr;
        int *cnt = nullptr;
        CK(c, lib_malloc((void **)&ent, (size_t)c->L.N * sizeof(uint2)));
        cudaError_t e = lib_malloc((void **)&cnt, sizeof(int));
        if (e != cudaSuccess) {
            cudaFree(ent);
            return cuda_fail(c, e, "add_particles: cudaMalloc(link list)");
        }
        CK(c, cudaMemset(cnt, 0, sizeof(int)));
        c->ll.ent = ent;
        c->ll.count = cnt;
        c->ll.cap = c->L.N;
        c->bytes += (size_t)c->L.N * sizeof(uint2) + sizeof(int);
    }
    {
        lbe_status cst = build_cells(c, blk, ncap, np);
        if (cst != LBE_OK) return cst;
    }
    if (ncap != cap) {
        double *nb = nullptr;
        float4 *nx32 = nullptr;
        double *npp = nullptr;
        void *ngeo = nullptr;
        CK(c, lib_malloc((void **)&nb, blk.size() * sizeof(double)));
        cudaError_t e = lib_malloc((void **)&nx32, x32.size() * sizeof(float4));
        if (e == cudaSuccess) e = lib_malloc((void **)&npp, (size_t)6 * ncap * sizeof(double));
        if (e == cudaSuccess) e = lib_malloc(&ngeo, (size_t)ncap * geom_bytes_per_particle());
        if (e != cudaSuccess) {
            cudaFree(nb);
            cudaFree(nx32);
            cudaFree(npp);
            return cuda_fail(c, e, "add_particles: cudaMalloc");
        }
        const size_t per_cap = PSTRIDE * sizeof(double) + 3 * sizeof(float4) + 6 * sizeof(double) +
                               geom_bytes_per_particle();
        if (c->pbuf) {
            cudaFree(c->pbuf);
            cudaFree(c->x32);
            cudaFree(c->ppart);
            cudaFree(c->geo);
            c->bytes -= (size_t)cap * per_cap;
        }
        c->pbuf = nb;
        c->x32 = nx32;
        c->ppart = npp;
        c->geo = ngeo;
        c->cap = ncap;
        c->bytes += (size_t)ncap * per_cap;
    }
    CK(c, cudaMemcpy(c->pbuf, blk.data(), blk.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(c, cudaMemcpy(c->x32, x32.data(), x32.size() * sizeof(float4), cudaMemcpyHostToDevice));
    c->np = np;
    c->L.np = np;
    bind_parts(c);
    drop_graphs(c);
    cudaStream_t s = c->stream;
    uint32_t *oo = c->owner[c->ocur], *on = c->owner[1 - c->ocur];
    launch_geom(c->L, c->P, s);
    launch_claim(c->L, c->P, 0, on, s);
    launch_transition(c->d.storage, c->L, c->P, c->f[c->cur], c->type, oo, on, 1, s);
    launch_reset(c->L, c->P, 1, oo, s);
    c->ocur = 1 - c->ocur;
    return sync(c, "add_particles");
}

lbe_status lbe_step(lbe_ctx *c, int32_t nsteps)
{
    if (!c || nsteps < 0) return LBE_EINVAL;
    cudaSetDevice(c->device);
    if (nsteps == 0) return LBE_OK;
    if (c->profiling) {
        for (int k = 0; k < nsteps; k++) enqueue_step(c);
        return check_async(c, "step");
    }
    int pairs = nsteps / 2;
    if (pairs > 0) {
        int key = c->cur * 2 + c->ocur;
        if (!c->graph[key]) {
            int cur0 = c->cur, ocur0 = c->ocur;
            cudaGraph_t g;
            CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            enqueue_step(c);
            enqueue_step(c);
            cudaError_t e = cudaStreamEndCapture(c->stream, &g);
            c->cur = cur0;
            c->ocur = ocur0;
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&c->graph[key], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
        }
        for (int k = 0; k < pairs; k++) CK(c, cudaGraphLaunch(c->graph[key], c->stream));
    }
    if (nsteps & 1) enqueue_step(c);
    return check_async(c, "step");
}

lbe_status lbe_read_fields(lbe_ctx *c, double *rho, double *vel, uint8_t *node_type)
{
    if (!c) return LBE_EINVAL;
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    const Lat &L = c->L;
    size_t N = (size_t)L.N;
    launch_moments(c->d.storage, L, c->f[c->cur], c->type, c->rho, c->psi, s);
    launch_shell(L, c->rho, c->psi, c->type, c->owner[c->ocur], c->P.drho, LinkList{nullptr, nullptr, 0}, s);
    double *dr = nullptr, *dv = nullptr;
    if (rho) CK(c, lib_malloc_async((void **)&dr, 2 * N * sizeof(double), s));
    if (vel) {
        cudaError_t e = lib_malloc_async((void **)&dv, 3 * N * sizeof(double), s);
        if (e != cudaSuccess) {
            if (dr) cudaFreeAsync(dr, s);
            return cuda_fail(c, e, "cudaMallocAsync(vel)");
        }
    }
    launch_fields(c->d.storage, L, c->f[c->cur], c->psi, c->type, dr, dv, s);
    if (rho) cudaMemcpyAsync(rho, dr, 2 * N * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (vel) cudaMemcpyAsync(vel, dv, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (node_type) cudaMemcpyAsync(node_type, c->type, N, cudaMemcpyDeviceToHost, s);
    if (dr) cudaFreeAsync(dr, s);
    if (dv) cudaFreeAsync(dv, s);
    return sync(c, "read_fields");
}

lbe_status lbe_read_particles(lbe_ctx *c, double *pos, double *quat, double *vel, double *omega,
                              double *force, double *torque)
{
    if (!c) return LBE_EINVAL;
    cudaSetDevice(c->device);
    lbe_status st = sync(c, "read_particles");
    if (st != LBE_OK || c->np == 0) return st;
    size_t cp = (size_t)c->cap;
    struct { double *dst; int off, k; } outs[] = {{pos, OX, 3}, {quat, OQ, 4}, {vel, OV, 3},
                                                  {omega, OW, 3}, {force, OF, 3}, {torque, OT, 3}};
    for (auto &o : outs)
        if (o.dst)
            CK(c, cudaMemcpy(o.dst, c->pbuf + (size_t)o.off * cp, (size_t)o.k * c->np * sizeof(double),
                             cudaMemcpyDeviceToHost));
    return LBE_OK;
}

lbe_status lbe_mass(lbe_ctx *c, double out[2])
{
    if (!c || !out) return LBE_EINVAL;
    cudaSetDevice(c->device);
    launch_mass(c->d.storage, c->L, c->f[c->cur], c->type, c->mass_partials, mass_blocks(), c->mass_out,
                c->stream);
    CK(c, cudaMemcpyAsync(out, c->mass_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    lbe_status st = sync(c, "mass");
    if (st != LBE_OK) return st;
    if (!std::isfinite(out[0]) || !std::isfinite(out[1]) || out[0] < 0 || out[1] < 0)
        return fail(c, LBE_ENUMERIC, "mass: non-finite or negative density");
    return LBE_OK;
}

lbe_status lbe_get_populations(lbe_ctx *c, double *f)
{
    if (!c || !f) return LBE_EINVAL;
    cudaSetDevice(c->device);
    size_t tot = (size_t)2 * Q * c->L.N;
    double *d = nullptr;
    CK(c, cudaMallocAsync((void **)&d, tot * sizeof(double), c->stream));
    launch_get_f(c->d.storage, c->L, c->f[c->cur], d, c->stream);
    cudaMemcpyAsync(f, d, tot * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(d, c->stream);
    return sync(c, "get_populations");
}

lbe_status lbe_set_populations(lbe_ctx *c, const double *f)
{
    if (!c || !f) return LBE_EINVAL;
    cudaSetDevice(c->device);
    size_t tot = (size_t)2 * Q * c->L.N;
    double *d = nullptr;
    CK(c, cudaMallocAsync((void **)&d, tot * sizeof(double), c->stream));
    cudaMemcpyAsync(d, f, tot * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    launch_set_f(c->d.storage, c->L, d, c->f[c->cur], c->stream);
    cudaFreeAsync(d, c->stream);
    return sync(c, "set_populations");
}

lbe_status lbe_profile_enable(lbe_ctx *c, int32_t enable)
{
    if (!c) return LBE_EINVAL;
    cudaSetDevice(c->device);
    lbe_status st = sync(c, "profile_enable");
    if (st != LBE_OK) return st;
    c->profiling = enable != 0;
    c->ev_used = 0;
    return LBE_OK;
}

lbe_status lbe_profile_read(lbe_ctx *c, double *ms_total, int64_t *launches)
{
    if (!c || !ms_total || !launches) return LBE_EINVAL;
    cudaSetDevice(c->device);
    lbe_status st = sync(c, "profile_read");
    if (st != LBE_OK) return st;
    double tot = 0.0;
    for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
        float ms = 0.f;
        CK(c, cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]));
        tot += ms;
    }
    *ms_total = tot;
    *launches = (int64_t)(c->ev_used / 2);
    return LBE_OK;
}

int32_t lbe_kernels_per_step(const lbe_ctx *c)
{
    if (!c) return 0;
    const bool two_pass = (c->d.flags & LBE_FLAG_TWO_PASS) != 0;
    // two-pass: densities, shell sweep, collide + stream; fused: the fused
    // kernel, with particles the densities and the shell fill per
    // particle, with walls the shell fill of the wall planes
    int k = 0;
    if (two_pass)
        k = 3;
    else
        k = 1 + (c->np > 0 ? 2 : 0) + (c->d.walls_z ? 1 : 0);
    if (c->np > 0) {
        k += 6;  // links, pair cells (count, prefix, fill), pairs, integrate
        if (c->d.particle_mode != LBE_PARTICLES_STATIC) k += 4;  // geometry, claim, transition, reset
    }
    return k;
}

size_t lbe_device_bytes(const lbe_ctx *c) { return c ? c->bytes : 0; }

size_t lbe_footprint(const lbe_lattice_desc *d, int32_t nparticles)
{
    if (!d || d->nx < 1 || d->ny < 1 || d->nz < 1 || nparticles < 0) return 0;
    if (d->storage < LBE_STORE_F32 || d->storage > LBE_STORE_F16_OFS) return 0;
    const size_t N = (size_t)d->nx * d->ny * d->nz;
    const size_t S = ((N + 127) / 128) * 128 + 384;
    size_t b = 2 * (size_t)2 * Q * S * storage_size(d->storage);  // two population buffers
    b += 2 * (2 * N * sizeof(float));                             // rho, psi
    b += N + 2 * N * 4;                                           // node types, two owner maps
    b += (size_t)2 * mass_blocks() * sizeof(double) + 2 * sizeof(double);
    b += 2 * N * sizeof(double);                                  // initial densities (transient)
    if (nparticles > 0) {
        const size_t cap = nparticles < 64 ? 64 : (size_t)nparticles + nparticles / 4;
        b += cap * (PSTRIDE * sizeof(double) + 3 * sizeof(float4) + 6 * sizeof(double) + 2 * sizeof(int) +
                    geom_bytes_per_particle());
        b += (3 * (N / 8) + 1) * sizeof(int);  // cells (at least 2 nodes a side)
        b += N * sizeof(uint2) + sizeof(int);  // link list
    }
    return b;
}

const char *lbe_last_error(const lbe_ctx *c) { return c ? c->err.c_str() : "null context"; }

void lbe_destroy(lbe_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

lbe_status lbe_autotune(lbe_ctx *c, int32_t *chosen_zc)
{
    if (!c) return LBE_EINVAL;
    cudaSetDevice(c->device);
    lbe_status st = sync(c, "autotune");
    if (st != LBE_OK) return st;
    if (c->d.flags & LBE_FLAG_TWO_PASS) {
        if (chosen_zc) *chosen_zc = 0;
        return LBE_OK;
    }
    // Candidates: tile heights (8, and 4 where built) times z chunks.
    // Each runs from the current populations into the spare buffer, which
    // the next step overwrites anyway, so the state is not changed.
    const Lat &L = c->L;
    std::vector<int> zcs;
    for (int zc = 4; zc < L.nz; zc *= 2) zcs.push_back(zc);
    zcs.push_back(L.nz);
    std::vector<int> tys = {8};
    if (fused_rows(L, 4, c->tma) == 4) tys.push_back(4);
    cudaEvent_t e0, e1;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    void *fin = c->f[c->cur], *fout = c->f[1 - c->cur];
    // ψ of the solid nodes, as the step's shell fill gives them
    launch_rho(c->d.storage, L, fin, c->type, c->rho, c->psi, c->stream);
    launch_shell(L, c->rho, c->psi, c->type, c->owner[c->ocur], c->P.drho, LinkList{nullptr, nullptr, 0}, c->stream);
    float best = 1e30f;
    int best_zc = 0, best_ty = 8;
    for (int ty : tys)
        for (int zc : zcs) {
            const CUtensorMap *tm = fused_map(c, c->cur, ty);
            const bool self = fused_self(c);
            launch_fused(c->d.storage, L, fin, fout, c->psi, c->type, tm, c->stream, zc, ty, FUSED_WAIT_LIMIT,
                         self);  // warm-up
            cudaEventRecord(e0, c->stream);
            for (int r = 0; r < 3; r++)
                launch_fused(c->d.storage, L, fin, fout, c->psi, c->type, tm, c->stream, zc, ty, FUSED_WAIT_LIMIT,
                             self);
            cudaEventRecord(e1, c->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_zc = zc;
                best_ty = ty;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->zc_tuned = best_zc;
    c->ty_tuned = best_ty;
    drop_graphs(c);
    if (chosen_zc) *chosen_zc = best_zc;
    return sync(c, "autotune");
}

lbe_status lbe_set_zchunk(lbe_ctx *c, int32_t zc)
{
    if (!c || zc < 0) return LBE_EINVAL;
    cudaSetDevice(c->device);
    lbe_status st = sync(c, "set_zchunk");  // no captured step in flight when its graph goes
    if (st != LBE_OK) return st;
    c->zc_tuned = zc < c->L.nz ? zc : c->L.nz;
    drop_graphs(c);
    return LBE_OK;
}

lbe_status lbe_set_tile(lbe_ctx *c, int32_t rows, int32_t zc)
{
    if (!c || (rows != 4 && rows != 8) || zc < 0) return LBE_EINVAL;
    cudaSetDevice(c->device);
    lbe_status st = sync(c, "set_tile");
    if (st != LBE_OK) return st;
    c->ty_tuned = rows;
    c->zc_tuned = zc < c->L.nz ? zc : c->L.nz;
    drop_graphs(c);
    return LBE_OK;
}

lbe_status lbe_get_tile(const lbe_ctx *c, int32_t *rows, int32_t *zc)
{
    if (!c || !rows || !zc) return LBE_EINVAL;
    if (c->d.flags & LBE_FLAG_TWO_PASS) {
        *rows = 0;
        *zc = 0;
        return LBE_OK;
    }
    *rows = fused_rows(c->L, c->ty_tuned, c->tma);
    *zc = c->zc_tuned > 0 ? c->zc_tuned : fused_zchunk(c->L, *rows);
    return LBE_OK;
}

void lbe_fail_allocations(int32_t after) { g_alloc_left.store(after < 0 ? -1 : after); }

lbe_status lbe_set_wait_limit(lbe_ctx *c, int32_t tries, int32_t unreachable)
{
    if (!c || tries < 0) return LBE_EINVAL;
    cudaSetDevice(c->device);
    lbe_status st = sync(c, "set_wait_limit");
    if (st != LBE_OK) return st;
    const int t = tries > 0 ? tries : FUSED_WAIT_LIMIT;
    c->wait_limit = unreachable ? -t : t;
    drop_graphs(c);
    return LBE_OK;
}

}  // extern "C"

// ----------------------------------------------------------------- batches

struct lbe_batch {
    std::vector<lbe_ctx *> members;   // in table order (largest box first)
    std::vector<int> order;           // table position -> position in the caller's list
    double *d_quat = nullptr, *h_quat = nullptr;  // first-particle orientations
    int device = 0, storage = 0;
    cudaStream_t stream = nullptr;    // the batch's own stream
    cudaEvent_t done = nullptr;       // end of the last batched launch
    std::vector<cudaEvent_t> mev;     // per member: its stream's last work
    BoxDev *d_box = nullptr;
    int *d_idx = nullptr;             // tile0 | node0 | part0 | par | counter
    BatchIndex idx{};
    int total_tiles = 0, total_nodes = 0, total_parts = 0;
    int ctas_per_sm = 0;
    cudaGraphExec_t graph = nullptr;
    std::string err;
};

namespace {

void batch_enqueue_step(lbe_batch *b)
{
    cudaStream_t s = b->stream;
    launch_rho_batch(b->storage, b->idx, b->total_nodes, s);
    launch_shell_batch(b->idx, b->total_nodes, s);
    cudaMemsetAsync(b->idx.counter, 0, sizeof(int), s);
    launch_fused_batch(b->storage, b->idx, b->total_tiles, 152 * b->ctas_per_sm, s);
    if (b->total_parts > 0) {
        launch_link_batch(b->storage, b->idx, s);
        launch_pairs_batch(b->idx, b->total_parts, s);
        launch_integrate_batch(b->idx, b->total_parts, s);
        launch_geom_batch(b->idx, b->total_parts, s);
        launch_claim_batch(b->idx, b->total_parts, s);
        launch_transition_batch(b->storage, b->idx, b->total_parts, s);
        launch_reset_batch(b->idx, b->total_parts, s);
    }
    launch_flip_batch(b->idx, s);
}

void batch_free(lbe_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (cudaEvent_t e : b->mev) cudaEventDestroy(e);
    cudaFree(b->d_quat);
    if (b->h_quat) cudaFreeHost(b->h_quat);
    if (b->done) cudaEventDestroy(b->done);
    if (b->stream) cudaStreamDestroy(b->stream);
    cudaFree(b->d_box);
    cudaFree(b->d_idx);
}

}  // namespace

extern "C" {

lbe_status lbe_batch_create(lbe_ctx *const *members, int32_t n, lbe_batch **out)
{
    if (!members || n < 1 || !out) return LBE_EINVAL;
    *out = nullptr;
    lbe_ctx *m0 = members[0];
    if (!m0) return LBE_EINVAL;
    for (int k = 0; k < n; k++) {
        lbe_ctx *c = members[k];
        if (!c || c->device != m0->device || c->d.storage != m0->d.storage) return LBE_EINVAL;
        if (c->d.flags & LBE_FLAG_TWO_PASS) return LBE_EINVAL;
        if (c->np > LBE_BATCH_MAX_PARTICLES) return LBE_EINVAL;
        if (n > 65535) return LBE_EINVAL;
        for (int j = 0; j < k; j++)
            if (members[j] == c) return LBE_EINVAL;
    }
    lbe_batch *b = new (std::nothrow) lbe_batch();
    if (!b) return LBE_ENOMEM;
    b->device = m0->device;
    b->storage = m0->d.storage;
    cudaSetDevice(b->device);
    std::vector<int> idx0(n);
    for (int k = 0; k < n; k++) {
        if (cudaStreamSynchronize(members[k]->stream) != cudaSuccess) {
            delete b;
            return LBE_ECUDA;
        }
        idx0[k] = k;
    }
    {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
        for (int k = 0; e == cudaSuccess && k < n; k++) {
            cudaEvent_t ev;
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) b->mev.push_back(ev);
        }
        if (e != cudaSuccess) {
            batch_free(b);
            delete b;
            return LBE_ECUDA;
        }
    }
    // largest boxes first, so that the persistent fused kernel starts on them
    std::stable_sort(idx0.begin(), idx0.end(),
                     [&](int x, int y) { return members[x]->L.N > members[y]->L.N; });
    for (int k = 0; k < n; k++) {
        b->members.push_back(members[idx0[k]]);
        b->order.push_back(idx0[k]);
    }
    std::vector<BoxDev> box(n);
    std::vector<int> idx(3 * (n + 1) + 2 * n + 1, 0);
    int *tile0 = idx.data(), *node0 = tile0 + (n + 1), *part0 = node0 + (n + 1), *par = part0 + (n + 1);
    for (int k = 0; k < n; k++) {
        lbe_ctx *c = b->members[k];
        BoxDev &d = box[k];
        d.L = c->L;
        d.ofs = fused_offsets(c->L);
        d.tma = c->tma ? 1 : 0;
        if (c->tma) {  // the batched kernel's tiles have FUSED_TY_BATCH = 8 rows
            d.tmap[0] = c->tmap[0][0][0];  // ψ from memory: the batch runs the density kernel
            d.tmap[1] = c->tmap[0][0][1];
        }
        d.f[0] = c->f[0];
        d.f[1] = c->f[1];
        d.rho = c->rho;
        d.psi = c->psi;
        d.type = c->type;
        d.owner[0] = c->owner[0];
        d.owner[1] = c->owner[1];
        d.P = c->P;
        d.P.n = c->np;
        d.pair = c->pair;
        d.mode = c->d.particle_mode;
        d.links = c->np > 0 ? c->ll : LinkList{nullptr, nullptr, 0};
        d.zc = c->zc_tuned > 0 ? c->zc_tuned : fused_zchunk(c->L, FUSED_TY_BATCH);
        d.ntx = (c->L.nx + FUSED_TX - 1) / FUSED_TX;
        d.nty = (c->L.ny + FUSED_TY_BATCH - 1) / FUSED_TY_BATCH;
        d.nzc = (c->L.nz + d.zc - 1) / d.zc;
        tile0[k + 1] = tile0[k] + d.ntx * d.nty * d.nzc;
        node0[k + 1] = node0[k] + c->L.N;
        part0[k + 1] = part0[k] + c->np;
        par[2 * k] = c->cur;
        par[2 * k + 1] = c->ocur;
    }
    b->total_tiles = tile0[n];
    b->total_nodes = node0[n];
    b->total_parts = part0[n];
    cudaError_t e = cudaMalloc((void **)&b->d_box, sizeof(BoxDev) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_idx, idx.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_quat, sizeof(double) * 4 * n);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_quat, sizeof(double) * 4 * n);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_box, box.data(), sizeof(BoxDev) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        batch_free(b);
        delete b;
        return e == cudaErrorMemoryAllocation ? LBE_ENOMEM : LBE_ECUDA;
    }
    b->idx.box = b->d_box;
    b->idx.nbox = n;
    b->idx.tile0 = b->d_idx;
    b->idx.node0 = b->d_idx + (n + 1);
    b->idx.part0 = b->d_idx + 2 * (n + 1);
    b->idx.par = b->d_idx + 3 * (n + 1);
    b->idx.counter = b->idx.par + 2 * n;
    b->ctas_per_sm = fused_batch_ctas_per_sm(b->storage);
    // link lists start empty; the last kernel of each batched step empties them
    for (lbe_ctx *c : b->members)
        if (c->np > 0 && c->ll.count) cudaMemsetAsync(c->ll.count, 0, sizeof(int), c->stream);
    for (lbe_ctx *c : b->members) cudaStreamSynchronize(c->stream);
    *out = b;
    return LBE_OK;
}

lbe_status lbe_batch_step(lbe_batch *b, int32_t nsteps)
{
    if (!b || nsteps < 0) return LBE_EINVAL;
    if (nsteps == 0) return LBE_OK;
    cudaSetDevice(b->device);
    if (!b->graph) {
        cudaGraph_t g;
        cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return LBE_ECUDA;
        batch_enqueue_step(b);
        e = cudaStreamEndCapture(b->stream, &g);
        if (e != cudaSuccess) return LBE_ECUDA;
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return LBE_ECUDA;
    }
    // order after the members' own work, and their later work after this
    for (size_t m = 0; m < b->members.size(); m++) {
        if (cudaEventRecord(b->mev[m], b->members[m]->stream) != cudaSuccess) return LBE_ECUDA;
        if (cudaStreamWaitEvent(b->stream, b->mev[m], 0) != cudaSuccess) return LBE_ECUDA;
    }
    for (int k = 0; k < nsteps; k++)
        if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return LBE_ECUDA;
    if (cudaEventRecord(b->done, b->stream) != cudaSuccess) return LBE_ECUDA;
    for (lbe_ctx *c : b->members)
        if (cudaStreamWaitEvent(c->stream, b->done, 0) != cudaSuccess) return LBE_ECUDA;
    // the members' host-side parities follow the device ones
    for (lbe_ctx *c : b->members) {
        if (nsteps & 1) {
            c->cur ^= 1;
            if (c->np > 0 && c->d.particle_mode != LBE_PARTICLES_STATIC) c->ocur ^= 1;
        }
    }
    return cudaGetLastError() == cudaSuccess ? LBE_OK : LBE_ECUDA;
}

lbe_status lbe_batch_autotune(lbe_batch *b, int32_t *chosen_ctas_per_sm)
{
    if (!b) return LBE_EINVAL;
    cudaSetDevice(b->device);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LBE_ECUDA;
    for (lbe_ctx *c : b->members)
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LBE_ECUDA;
    // Persistent CTAs per SM for the batched fused kernel, timed on the
    // fused kernel alone (it writes only the spare buffers; the link sums it
    // accumulates are cleared afterwards).
    const int maxc = fused_batch_ctas_per_sm(b->storage);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_c = maxc;
    for (int cps = 1; cps <= maxc; cps++) {
        for (int r = 0; r < 4; r++) {
            if (r == 1) cudaEventRecord(e0, b->stream);
            cudaMemsetAsync(b->idx.counter, 0, sizeof(int), b->stream);
            launch_fused_batch(b->storage, b->idx, b->total_tiles, 152 * cps, b->stream);
        }
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_c = cps;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (lbe_ctx *c : b->members)
        if (c->np > 0) cudaMemsetAsync(c->P.fix, 0, (size_t)6 * c->np * sizeof(unsigned long long), b->stream);
    b->ctas_per_sm = best_c;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (chosen_ctas_per_sm) *chosen_ctas_per_sm = best_c;
    return cudaStreamSynchronize(b->stream) == cudaSuccess ? LBE_OK : LBE_ECUDA;
}

lbe_status lbe_batch_first_quat(lbe_batch *b, double *quat_out)
{
    if (!b || !quat_out) return LBE_EINVAL;
    cudaSetDevice(b->device);
    launch_batch_quat(b->idx, b->d_quat, b->stream);
    const size_t n = b->members.size();
    if (cudaMemcpyAsync(b->h_quat, b->d_quat, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
        return LBE_ECUDA;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LBE_ECUDA;
    for (size_t k = 0; k < n; k++)
        for (int j = 0; j < 4; j++) quat_out[4 * b->order[k] + j] = b->h_quat[4 * k + j];
    return LBE_OK;
}

int32_t lbe_batch_kernels_per_step(const lbe_batch *b)
{
    if (!b) return 0;
    return b->total_parts > 0 ? 11 : 4;
}

void lbe_batch_destroy(lbe_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_free(b);
    delete b;
}

}  // extern "C"
