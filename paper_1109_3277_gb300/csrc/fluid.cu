// Fluid kernels of the lattice Boltzmann step (§2 of Günther et al.,
// arXiv:1109.3277): moments, ψ, outer-shell fill with the colour rule,
// Shan–Chen force (Eq. 3), shifted-velocity BGK collision (Eq. 2) and
// streaming (Eq. 1) with halfway bounce-back, plus readers and mass sums.
#include "lbe_internal.cuh"

namespace lbe {

namespace {

struct Coord {
    int x, y, z;
};

__device__ __forceinline__ Coord coord_of(const Lat &L, int n)
{
    Coord c;
    c.x = n % L.nx;
    int t = n / L.nx;
    c.y = t % L.ny;
    c.z = t / L.ny;
    return c;
}

// Wrapped coordinates x-1, x, x+1 (and for y, z).  With walls the z
// neighbours of the boundary planes do not exist and are flagged -1.
struct Nbr {
    int xs[3], ys[3], zs[3];
};

__device__ __forceinline__ Nbr nbr_of(const Lat &L, Coord c)
{
    Nbr b;
    b.xs[0] = c.x == 0 ? L.nx - 1 : c.x - 1;
    b.xs[1] = c.x;
    b.xs[2] = c.x == L.nx - 1 ? 0 : c.x + 1;
    b.ys[0] = c.y == 0 ? L.ny - 1 : c.y - 1;
    b.ys[1] = c.y;
    b.ys[2] = c.y == L.ny - 1 ? 0 : c.y + 1;
    if (L.walls) {
        b.zs[0] = c.z - 1;
        b.zs[2] = c.z + 1 < L.nz ? c.z + 1 : -1;
    } else {
        b.zs[0] = c.z == 0 ? L.nz - 1 : c.z - 1;
        b.zs[2] = c.z == L.nz - 1 ? 0 : c.z + 1;
    }
    b.zs[1] = c.z;
    return b;
}

__device__ __forceinline__ int nidx(const Lat &L, const Nbr &b, int i)
{
    int z = b.zs[cz(i) + 1];
    if (z < 0) return -1;
    return b.xs[cx(i) + 1] + L.nx * (b.ys[cy(i) + 1] + L.ny * z);
}

// ---------------------------------------------------------------- init

template <class S>
__global__ void k_init_f(Lat L, const double *__restrict__ rho0, typename S::P *__restrict__ f,
                         const uint8_t *__restrict__ type)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= L.N) return;
    bool fl = type[n] == FLUID;
    const float r0 = fl ? (float)rho0[n] : 0.f, r1 = fl ? (float)rho0[(size_t)L.N + n] : 0.f;
#pragma unroll
    for (int i = 0; i < Q; i++) st2f<S>(f, L, i, n, make_float2(wgt(i) * r0, wgt(i) * r1));
}

// ------------------------------------------------------------- moments
// ρ^c = Σ_i f_i^c on fluid nodes and ψ^c = 1 - exp(-ρ^c) (Eq. 3's weight).

template <class S>
__global__ void __launch_bounds__(256) k_moments(Lat L, const typename S::P *__restrict__ f,
                                                 const uint8_t *__restrict__ type,
                                                 float *__restrict__ rho, float *__restrict__ psi)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= L.N || type[n] != FLUID) return;
    float r0 = 0.f, r1 = 0.f;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const float2 v = ld2f<S>(f, L, i, n);
        r0 += v.x;
        r1 += v.y;
    }
    st_pair(rho, n, make_float2(r0, r1));
    psi[n] = 1.f - expf(-r0);
    psi[(size_t)L.N + n] = 1.f - expf(-r1);
}

// ------------------------------------------------------------ densities
// ρ^c = Σ_i f_i^c on every fluid node, for the shell fill and the link
// kernel, and ψ^c = 1 - exp(-ρ^c) for the fused kernel (which sums its own
// nodes' stored populations in the same order and adds ρ_ref the same way,
// so the two agree bit for bit; the shell fill writes ψ of the solid nodes
// into the same array).  One thread per node: each pair load brings both
// components of a direction.

template <class S>
__global__ void __launch_bounds__(256) k_rho(Lat L, const typename S::P *__restrict__ f,
                                             const uint8_t *__restrict__ type, float *__restrict__ rho,
                                             float *__restrict__ psi)
{
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= L.N || type[n] != FLUID) return;
    const float2 r = node_rho2<S>(f, L, n);
    st_pair(rho, n, r);
    psi[n] = 1.f - expf(-r.x);
    psi[(size_t)L.N + n] = 1.f - expf(-r.y);
}

// Neighbour indexing on a 3D grid (x per thread, one y row and z plane per
// block row): no index division, and interior nodes reach their neighbours
// by a fixed offset.

__device__ __forceinline__ int nb_off(const Lat &L, int i) { return cx(i) + L.nx * (cy(i) + L.ny * cz(i)); }

struct Site {
    int x, y, z, n;
    bool inner;
};

__device__ __forceinline__ bool site_of(const Lat &L, Site &s)
{
    s.x = blockIdx.x * blockDim.x + threadIdx.x;
    s.y = blockIdx.y;
    s.z = blockIdx.z;
    if (s.x >= L.nx) return false;
    s.n = s.x + L.nx * (s.y + L.ny * s.z);
    s.inner = s.x >= 1 && s.x <= L.nx - 2 && s.y >= 1 && s.y <= L.ny - 2 && s.z >= 1 && s.z <= L.nz - 2;
    return true;
}

__device__ __forceinline__ int site_nb(const Lat &L, const Site &s, int i)
{
    if (s.inner) return s.n + nb_off(L, i);
    Coord c{s.x, s.y, s.z};
    Nbr b = nbr_of(L, c);
    return nidx(L, b, i);
}

// Batched form: lanes may belong to different boxes (key: the box, or -1
// for a lane without a node); lanes of the same box share one atomic on the
// box's counter.  Called by all 32 lanes.
__device__ __forceinline__ void append_links_keyed(const LinkList &ll, int key, int n, uint32_t m)
{
    if (!__any_sync(0xffffffffu, m != 0)) return;
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    const unsigned want = __ballot_sync(0xffffffffu, m != 0) & grp;
    const int lane = threadIdx.x & 31;
    const int leader = want ? __ffs(want) - 1 : lane;
    int base = 0;
    if (want && lane == leader) base = atomicAdd(ll.count, __popc(want));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (m) {
        const int k = base + __popc(want & ((1u << lane) - 1u));
        if (k < ll.cap) ll.ent[k] = make_uint2((unsigned)n, m);
    }
}

// Node g of a batch (all boxes' nodes in box order) as a site of its box.
__device__ __forceinline__ const BoxDev &batch_site(const BatchIndex &B, int g, Site &s)
{
    const int b = find_box(B.node0, B.nbox, g);
    const BoxDev &bx = B.box[b];
    const int n = g - B.node0[b];
    s.n = n;
    s.x = n % bx.L.nx;
    const int t = n / bx.L.nx;
    s.y = t % bx.L.ny;
    s.z = t / bx.L.ny;
    s.inner = s.x >= 1 && s.x <= bx.L.nx - 2 && s.y >= 1 && s.y <= bx.L.ny - 2 && s.z >= 1 && s.z <= bx.L.nz - 2;
    return bx;
}

// Densities of the fluid nodes of all boxes, one node per thread (batched
// boxes are small).
template <class S>
__global__ void __launch_bounds__(256) k_rho_batch(BatchIndex B, int total)
{
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        Site s;
        const BoxDev &bx = batch_site(B, g, s);
        if (bx.type[s.n] != FLUID) continue;
        const int b = find_box(B.node0, B.nbox, g);
        const typename S::P *f = (const typename S::P *)bx.f[B.par[2 * b]];
        const float2 r = node_rho2<S>(f, bx.L, s.n);
        st_pair(bx.rho, s.n, r);
        bx.psi[s.n] = 1.f - expf(-r.x);
        bx.psi[(size_t)bx.L.N + s.n] = 1.f - expf(-r.y);
    }
}

// ---------------------------------------------------------- shell fill
// Solid nodes with at least one fluid neighbour take the mean ρ^c of those
// neighbours (Eq. 10); the colour Δρ of the owning particle is added to red
// if positive, else |Δρ| to blue.  Walls take Δρ = 0.  A particle node
// among them returns the mask of its fluid neighbours (its links), 0
// otherwise.

__device__ __forceinline__ uint32_t shell_node(const Lat &L, const float *__restrict__ rho, float *__restrict__ psi,
                                               const uint8_t *__restrict__ type, const uint32_t *__restrict__ owner,
                                               const double *__restrict__ drho, const Site &s)
{
    const uint8_t t = type[s.n];
    if (t == FLUID) return 0;
    float dr = 0.f;
    if (t == PART) {
        uint32_t o = owner[s.n];
        if (idx_ok(L, o, L.np, 1)) dr = (float)drho[o];
    }
    const uint32_t fm = shell_fill(L, rho, psi, type, s.n, dr, [&](int i) { return site_nb(L, s, i); });
    return t == PART ? fm : 0u;
}

__global__ void __launch_bounds__(128) k_shell(Lat L, const float *__restrict__ rho, float *__restrict__ psi,
                                               const uint8_t *__restrict__ type, const uint32_t *__restrict__ owner,
                                               const double *__restrict__ drho, LinkList ll)
{
    Site s{};
    const bool valid = site_of(L, s);
    const uint32_t fm = valid ? shell_node(L, rho, psi, type, owner, drho, s) : 0u;
    if (ll.ent) append_links(ll, s.n, fm);
}

__global__ void __launch_bounds__(256) k_shell_batch(BatchIndex B, int total)
{
    // warp-uniform trip count: every lane takes part in the appends
    const int stride = gridDim.x * blockDim.x;
    for (int w0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < total; w0 += stride) {
        const int g = w0 + (threadIdx.x & 31);
        int key = -1, n = 0;
        uint32_t fm = 0;
        LinkList ll{nullptr, nullptr, 0};
        if (g < total) {
            Site s;
            const BoxDev &bx = batch_site(B, g, s);
            const int b = find_box(B.node0, B.nbox, g);
            fm = shell_node(bx.L, bx.rho, bx.psi, bx.type, bx.owner[B.par[2 * b + 1]], bx.P.drho, s);
            ll = bx.links;
            if (ll.ent)
                key = b;
            else
                fm = 0;
            n = s.n;
        }
        append_links_keyed(ll, key, n, fm);
    }
}

// ------------------------------------------------------ collide + stream
// Shan–Chen force F^c = -g ψ^c(x) Σ_{i=1..18} ψ^{c'}(x+c_i) c_i + ρ^c g_body,
// shifted velocity u' = Σ_c j^c/τ_c / Σ_c ρ^c/τ_c, equilibrium of component
// c at u' + τ_c F^c/ρ^c, BGK relaxation, then push streaming: a population
// whose target is solid is reflected into the opposite slot of its own node.

template <class S>
__global__ void __launch_bounds__(256) k_collide_stream(Lat L, const typename S::P *__restrict__ fin,
                                                        typename S::P *__restrict__ fout,
                                                        const float *__restrict__ psi,
                                                        const uint8_t *__restrict__ type)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= L.N || type[n] != FLUID) return;
    Coord co = coord_of(L, n);
    Nbr b = nbr_of(L, co);
    float f[2][Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const float2 v = ld2f<S>(fin, L, i, n);
        f[0][i] = v.x;
        f[1][i] = v.y;
    }
    float rho[2], j[2][3];
#pragma unroll
    for (int c = 0; c < 2; c++) {
        float r = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            r += f[c][i];
            if (cx(i)) jx += cx(i) * f[c][i];
            if (cy(i)) jy += cy(i) * f[c][i];
            if (cz(i)) jz += cz(i) * f[c][i];
        }
        rho[c] = r;
        j[c][0] = jx;
        j[c][1] = jy;
        j[c][2] = jz;
    }
    float s[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    int nb[Q];
#pragma unroll
    for (int i = 1; i < Q; i++) {
        int m = nidx(L, b, i);
        nb[i] = m;
        float p0 = m >= 0 ? psi[m] : 0.f, p1 = m >= 0 ? psi[(size_t)L.N + m] : 0.f;
        // red feels blue's ψ and vice versa
        if (cx(i)) { s[0][0] += cx(i) * p1; s[1][0] += cx(i) * p0; }
        if (cy(i)) { s[0][1] += cy(i) * p1; s[1][1] += cy(i) * p0; }
        if (cz(i)) { s[0][2] += cz(i) * p1; s[1][2] += cz(i) * p0; }
    }
    nb[0] = n;
    float den = rho[0] * L.itau[0] + rho[1] * L.itau[1];
    float up[3];
#pragma unroll
    for (int k = 0; k < 3; k++)
        up[k] = den > 0.f ? (j[0][k] * L.itau[0] + j[1][k] * L.itau[1]) / den : 0.f;
    bool solid_nb[Q];
#pragma unroll
    for (int i = 1; i < Q; i++) solid_nb[i] = nb[i] < 0 || type[nb[i]] != FLUID;
    float fs[2][Q];
#pragma unroll
    for (int c = 0; c < 2; c++) {
        float pc = psi[(size_t)c * L.N + n];
        float r = rho[c];
        float ue[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            float F = -L.g * pc * s[c][k] + r * L.body[k];
            ue[k] = r > 0.f ? up[k] + L.tau[c] * F / r : up[k];
        }
        float uu = ue[0] * ue[0] + ue[1] * ue[1] + ue[2] * ue[2];
        float it = L.itau[c];
        // The rest equilibrium is taken as ρ - Σ_{i>0} f^eq_i, equal to the
        // formula in exact arithmetic; in FP32 it keeps Σ f^eq = ρ free of
        // the systematic error of the rounded weights (Σ w_i = 1 + 1.5e-8).
        float seq = 0.f;
#pragma unroll
        for (int i = 1; i < Q; i++) {
            float cu = cx(i) * ue[0] + cy(i) * ue[1] + cz(i) * ue[2];
            float feq = wgt(i) * r * (1.f + 3.f * cu + 4.5f * cu * cu - 1.5f * uu);
            seq += feq;
            fs[c][i] = f[c][i] - (f[c][i] - feq) * it;
        }
        fs[c][0] = f[c][0] - (f[c][0] - (r - seq)) * it;
    }
    // push both components of each direction: to the neighbour, or reflected
    // into the opposite slot of this node (same weight, same base)
#pragma unroll
    for (int i = 1; i < Q; i++) {
        const float2 v = make_float2(fs[0][i], fs[1][i]);
        if (!solid_nb[i])
            st2f<S>(fout, L, i, nb[i], v);
        else
            st2f<S>(fout, L, opp(i), n, v);
    }
    st2f<S>(fout, L, 0, n, make_float2(fs[0][0], fs[1][0]));
}

// -------------------------------------------------------------- fields

template <class S>
__global__ void k_fields(Lat L, const typename S::P *__restrict__ f, const float *__restrict__ psi,
                         const uint8_t *__restrict__ type, double *__restrict__ rho_out,
                         double *__restrict__ vel_out)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= L.N) return;
    if (type[n] != FLUID) {
        if (rho_out) {
            rho_out[n] = 0.0;
            rho_out[(size_t)L.N + n] = 0.0;
        }
        if (vel_out)
            for (int k = 0; k < 3; k++) vel_out[(size_t)k * L.N + n] = 0.0;
        return;
    }
    Coord co = coord_of(L, n);
    Nbr b = nbr_of(L, co);
    float rho[2] = {0.f, 0.f}, m[3] = {0.f, 0.f, 0.f};
    for (int c = 0; c < 2; c++) {
        for (int i = 0; i < Q; i++) {
            const float2 v2 = ld2f<S>(f, L, i, n);
            const float v = c ? v2.y : v2.x;
            rho[c] += v;
            m[0] += cx(i) * v;
            m[1] += cy(i) * v;
            m[2] += cz(i) * v;
        }
    }
    for (int c = 0; c < 2; c++) {
        float sx = 0.f, sy = 0.f, sz = 0.f;
        for (int i = 1; i < Q; i++) {
            int mm = nidx(L, b, i);
            float p = mm >= 0 ? psi[(size_t)(1 - c) * L.N + mm] : 0.f;
            sx += cx(i) * p;
            sy += cy(i) * p;
            sz += cz(i) * p;
        }
        float pc = psi[(size_t)c * L.N + n];
        m[0] += 0.5f * (-L.g * pc * sx + rho[c] * L.body[0]);
        m[1] += 0.5f * (-L.g * pc * sy + rho[c] * L.body[1]);
        m[2] += 0.5f * (-L.g * pc * sz + rho[c] * L.body[2]);
    }
    float tot = rho[0] + rho[1];
    if (rho_out) {
        rho_out[n] = rho[0];
        rho_out[(size_t)L.N + n] = rho[1];
    }
    if (vel_out)
        for (int k = 0; k < 3; k++) vel_out[(size_t)k * L.N + n] = tot > 0.f ? m[k] / tot : 0.0;
}

// ---------------------------------------------------------------- mass
// Per-block FP64 partial sums in a fixed grid-stride order, then one block
// adds the partials in index order: the result does not depend on timing.

constexpr int MASS_BLOCKS = 1024;
constexpr int MASS_THREADS = 256;

// Σ_i f_i^c of node n.  The 19 FP32 values are added with Knuth's
// error-free TwoSum: s collects the rounded sum and e the rounding errors,
// so s + e is the exact sum up to the rounding of the small term e (about
// 1e-15 of the node's mass), and only two FP64 additions per node and
// component remain (FP64 arithmetic is slow on this part).
__device__ __forceinline__ void two_sum_acc(float &s, float &e, float v)
{
    const float t = __fadd_rn(s, v);
    const float vb = __fsub_rn(t, s);
    e = __fadd_rn(e, __fadd_rn(__fsub_rn(s, __fsub_rn(t, vb)), __fsub_rn(v, vb)));
    s = t;
}

template <class S>
__device__ __forceinline__ void node_mass(const Lat &L, const typename S::P *__restrict__ f, long long n, double &m0,
                                          double &m1)
{
    const float2 v0 = ld2f<S>(f, L, 0, n);
    float s0 = v0.x, s1 = v0.y, e0 = 0.f, e1 = 0.f;
#pragma unroll
    for (int i = 1; i < Q; i++) {
        const float2 v = ld2f<S>(f, L, i, n);
        two_sum_acc(s0, e0, v.x);
        two_sum_acc(s1, e1, v.y);
    }
    m0 = (double)s0 + (double)e0;
    m1 = (double)s1 + (double)e1;
}

// The grid-stride index is 64-bit: N may come within a stride of 2^31 - 1.
template <class S>
__global__ void __launch_bounds__(MASS_THREADS) k_mass(Lat L, const typename S::P *__restrict__ f,
                                                       const uint8_t *__restrict__ type,
                                                       double *__restrict__ partials)
{
    double a0 = 0.0, a1 = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < L.N; n += stride) {
        if (type[n] != FLUID) continue;
        double m0, m1;
        node_mass<S>(L, f, n, m0, m1);
        a0 += m0;
        a1 += m1;
    }
    __shared__ double sh[2][MASS_THREADS];
    sh[0][threadIdx.x] = a0;
    sh[1][threadIdx.x] = a1;
    __syncthreads();
    for (int w = MASS_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = sh[0][0];
        partials[gridDim.x + blockIdx.x] = sh[1][0];
    }
}

__global__ void k_mass_final(const double *__restrict__ partials, int nb, double *__restrict__ out)
{
    __shared__ double sh[2][MASS_THREADS];
    double a0 = 0.0, a1 = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        a0 += partials[k];
        a1 += partials[nb + k];
    }
    sh[0][threadIdx.x] = a0;
    sh[1][threadIdx.x] = a1;
    __syncthreads();
    for (int w = MASS_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sh[0][0];
        out[1] = sh[1][0];
    }
}

// --------------------------------------------------------- raw f access

// The caller's layout is [2][19][N]; element (c, i, n) of the device
// array is scalar 2 (i S + n) + c.
template <class S>
__global__ void k_get_f(Lat L, const typename S::T *__restrict__ f, double *__restrict__ out)
{
    size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t tot = (size_t)2 * Q * L.N;
    if (k >= tot) return;
    int ci = (int)(k / L.N);
    size_t n = k - (size_t)ci * L.N;
    const int c = ci / Q, i = ci % Q;
    out[k] = (double)(L.base[c][i] + S::raw(f[2 * pidx(L, i, (long long)n) + c]));
}

template <class S>
__global__ void k_set_f(Lat L, const double *__restrict__ in, typename S::T *__restrict__ f)
{
    size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t tot = (size_t)2 * Q * L.N;
    if (k >= tot) return;
    int ci = (int)(k / L.N);
    size_t n = k - (size_t)ci * L.N;
    const int c = ci / Q, i = ci % Q;
    f[2 * pidx(L, i, (long long)n) + c] = S::enc((float)in[k] - L.base[c][i]);
}

inline unsigned blocks_for(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int mass_blocks() { return MASS_BLOCKS; }

#define LBE_DISPATCH(storage, CALL)                  \
    do {                                             \
        switch (storage) {                           \
        case LBE_STORE_F16_OFS: { using S = StF16; CALL; } break;  \
        case LBE_STORE_BF16_OFS: { using S = StBF16; CALL; } break; \
        default: { using S = StF32; CALL; } break;   \
        }                                            \
    } while (0)

void launch_init_f(int storage, const Lat &L, const double *rho0, void *f, const uint8_t *type,
                   cudaStream_t s)
{
    LBE_DISPATCH(storage, (k_init_f<S><<<blocks_for(L.N, 256), 256, 0, s>>>(
                              L, rho0, (typename S::P *)f, type)));
}

void launch_moments(int storage, const Lat &L, const void *f, const uint8_t *type, float *rho,
                    float *psi, cudaStream_t s)
{
    LBE_DISPATCH(storage, (k_moments<S><<<blocks_for(L.N, 256), 256, 0, s>>>(
                              L, (const typename S::P *)f, type, rho, psi)));
}

void launch_rho(int storage, const Lat &L, const void *f, const uint8_t *type, float *rho, float *psi,
                cudaStream_t s)
{
    LBE_DISPATCH(storage,
                 (k_rho<S><<<blocks_for(L.N, 256), 256, 0, s>>>(L, (const typename S::P *)f, type, rho, psi)));
}

static unsigned batch_grid(int total)
{
    unsigned g = (unsigned)((total + 255) / 256);
    return g > 8 * 152 ? 8 * 152 : (g ? g : 1);
}

void launch_rho_batch(int storage, const BatchIndex &B, int total_nodes, cudaStream_t s)
{
    LBE_DISPATCH(storage, (k_rho_batch<S><<<batch_grid(total_nodes), 256, 0, s>>>(B, total_nodes)));
}

void launch_shell_batch(const BatchIndex &B, int total_nodes, cudaStream_t s)
{
    k_shell_batch<<<batch_grid(total_nodes), 256, 0, s>>>(B, total_nodes);
}

void launch_shell(const Lat &L, const float *rho, float *psi, const uint8_t *type, const uint32_t *owner,
                  const double *drho, const LinkList &ll, cudaStream_t s)
{
    dim3 grid((L.nx + 127) / 128, L.ny, L.nz);
    k_shell<<<grid, 128, 0, s>>>(L, rho, psi, type, owner, drho, ll);
}

void launch_collide_stream(int storage, const Lat &L, const void *fin, void *fout, const float *psi,
                           const uint8_t *type, cudaStream_t s)
{
    LBE_DISPATCH(storage, (k_collide_stream<S><<<blocks_for(L.N, 256), 256, 0, s>>>(
                              L, (const typename S::P *)fin, (typename S::P *)fout, psi, type)));
}

void launch_fields(int storage, const Lat &L, const void *f, const float *psi, const uint8_t *type,
                   double *rho_out, double *vel_out, cudaStream_t s)
{
    LBE_DISPATCH(storage, (k_fields<S><<<blocks_for(L.N, 256), 256, 0, s>>>(
                              L, (const typename S::P *)f, psi, type, rho_out, vel_out)));
}

void launch_mass(int storage, const Lat &L, const void *f, const uint8_t *type, double *partials,
                 int nblocks, double *out, cudaStream_t s)
{
    LBE_DISPATCH(storage, (k_mass<S><<<nblocks, MASS_THREADS, 0, s>>>(
                              L, (const typename S::P *)f, type, partials)));
    k_mass_final<<<1, MASS_THREADS, 0, s>>>(partials, nblocks, out);
}

void launch_get_f(int storage, const Lat &L, const void *f, double *out, cudaStream_t s)
{
    size_t tot = (size_t)2 * Q * L.N;
    LBE_DISPATCH(storage, (k_get_f<S><<<blocks_for(tot, 256), 256, 0, s>>>(
                              L, (const typename S::T *)f, out)));
}

void launch_set_f(int storage, const Lat &L, const double *in, void *f, cudaStream_t s)
{
    size_t tot = (size_t)2 * Q * L.N;
    LBE_DISPATCH(storage, (k_set_f<S><<<blocks_for(tot, 256), 256, 0, s>>>(
                              L, in, (typename S::T *)f)));
}

}  // namespace lbe
