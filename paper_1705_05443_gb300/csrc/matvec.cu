// matvec.cu -- the node-wise H^2 matvec of Section 3.4 in FP64:
//   gather q into Morton order, near field over L^- (3.20), upward pass
//   q^_i = V_i^T q | sum_c W_c^T q^_c, coupling over L with the kernel
//   evaluated on skeleton pairs (3.19), downward pass z^_c += R_c z^_i and
//   z|_i += U_i z^_i, scatter back to the caller's order.
// The transfer matrices are used in their ID form [I; G] (2.11): the
// identity rows are copies, only G is multiplied.
#include <algorithm>
#include <cmath>

#include "internal.cuh"
#include "ksum_tiles.cuh"

namespace smash {

// ------------------------------------------------------------------ kernels kappa
template <int KID>
__device__ __forceinline__ double kappa64(double dx, double dy, double dz) {
    if (KID == SMASH_K_CAUCHY1D) return dx != 0.0 ? 1.0 / dx : 0.0;
    double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0) return 0.0;
    // y-gradient of -(1/2pi) log|x - y| with d = x - y: d_a / (2 pi |d|^2)
    if (KID == SMASH_K_DLP1) return dx / (6.283185307179586 * r2);
    if (KID == SMASH_K_DLP2) return dy / (6.283185307179586 * r2);
    if (KID == SMASH_K_INVR) return rsqrt(r2);
    if (KID == SMASH_K_LOG) return 0.5 * log(r2);
    double r = sqrt(r2);
    return exp(-r) / r;  // SMASH_K_YUKAWA
}

// ------------------------------------------------------------------ gather / scatter
__global__ void gather_rhs_kernel(const double *__restrict__ X, int nrhs, const int64_t *__restrict__ perm,
                                  int64_t n, int ldq, double *__restrict__ qs) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * ldq) return;
    int64_t p = i / ldq;
    int c = (int)(i % ldq);
    qs[i] = c < nrhs ? X[perm[p] * nrhs + c] : 0.0;
}

__global__ void scatter_rhs_kernel(const double *__restrict__ zs, int ldq, const int64_t *__restrict__ perm,
                                   int64_t n, int nrhs, double *__restrict__ Y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nrhs) return;
    int64_t p = i / nrhs;
    int c = (int)(i % nrhs);
    Y[perm[p] * nrhs + c] = zs[p * ldq + c];
}

// ------------------------------------------------------------------ transfers
struct PassArgs {
    int64_t n0;
    const int32_t *leaf, *m, *k;
    const int64_t *in_off, *sk_off, *loc_off, *g_off;
    const int32_t *loc;
    const double *G;
    const double *pts_vec;   // leaf-level vectors (qs or zs), ldq
    double *skel_vec_in;     // skeleton vectors read (qhat, or zhat)
    double *skel_vec_out;    // skeleton vectors written (qhat, or zhat of children)
    double *pts_vec_out;     // zs for leaves in the downward pass
    int ldq;
};

// q^_i[t] = x[skel_t] + sum_u G[u][t] x[rest_u],  x = q|_i (leaf) or [q^_c] (parent)
__global__ void __launch_bounds__(256) upward_kernel(PassArgs a) {
    const int64_t g = a.n0 + blockIdx.x;
    const int m = a.m[g], k = a.k[g];
    if (k == 0) return;
    const int ldq = a.ldq;
    const double *in = a.leaf[g] ? a.pts_vec + a.in_off[g] * ldq : a.skel_vec_in + a.in_off[g] * ldq;
    const int32_t *loc = a.loc + a.loc_off[g];
    const double *G = a.G + a.g_off[g];
    double *out = a.skel_vec_out + a.sk_off[g] * ldq;
    const int mk = m - k;
    for (int e = threadIdx.x; e < k * ldq; e += blockDim.x) {
        int t = e / ldq, c = e % ldq;
        double s = in[(int64_t)loc[t] * ldq + c];
        for (int u = 0; u < mk; ++u) s += G[(int64_t)u * k + t] * in[(int64_t)loc[k + u] * ldq + c];
        out[(int64_t)t * ldq + c] = s;
    }
}

// out[skel_t] += z^_i[t];  out[rest_u] += sum_t G[u][t] z^_i[t]
__global__ void __launch_bounds__(256) downward_kernel(PassArgs a) {
    const int64_t g = a.n0 + blockIdx.x;
    const int m = a.m[g], k = a.k[g];
    if (k == 0) return;
    const int ldq = a.ldq;
    const double *zin = a.skel_vec_in + a.sk_off[g] * ldq;
    double *out = a.leaf[g] ? a.pts_vec_out + a.in_off[g] * ldq : a.skel_vec_out + a.in_off[g] * ldq;
    const int32_t *loc = a.loc + a.loc_off[g];
    const double *G = a.G + a.g_off[g];
    for (int e = threadIdx.x; e < m * ldq; e += blockDim.x) {
        int row = e / ldq, c = e % ldq;
        double s;
        if (row < k) {
            s = zin[(int64_t)row * ldq + c];
        } else {
            const double *gr = G + (int64_t)(row - k) * k;
            s = 0.0;
            for (int t = 0; t < k; ++t) s += gr[t] * zin[(int64_t)t * ldq + c];
        }
        out[(int64_t)loc[row] * ldq + c] += s;
    }
}

// ------------------------------------------------------------------ kernel sums
// out[t_off(g) + a] = sum over partners j of g in the CSR, over the points b
// of j:  kappa(x_a, y_b) q[s_off(j) + b].  Used for the coupling (targets and
// sources are skeleton slots) and for the near field (sorted points).
struct KsumArgs {
    const int32_t *tnodes;
    const int64_t *t_off;
    const int32_t *t_cnt;
    const int64_t *ptr;
    const int32_t *col;
    const int64_t *s_off;
    const int32_t *s_cnt;
    const double *xt;  // target coordinates, stride 4
    const double *ys;  // source coordinates, stride 4
    const double *qv;  // source vectors, ldq
    double *out;       // target vectors, ldq
    int ldq, nchunks, tbp, groups;
    int tile;          // source points staged per round (<= kKsTile)
};

constexpr int kKsThreads = 256;
constexpr int kKsTile = 128;  // source points staged per round

template <int KID, int RC>
__global__ void __launch_bounds__(kKsThreads) ksum_f64_kernel(KsumArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ PartnerChunk pc;
    const int tile = a.tile;                                   // <= kKsTile
    P4 *sy = reinterpret_cast<P4 *>(smraw);                     // tile
    double *sq = reinterpret_cast<double *>(sy + tile);                   // tile * ldq
    double *red = sq + (size_t)tile * a.ldq;                             // tbp * ldq
    int64_t *sidx = reinterpret_cast<int64_t *>(red + (size_t)a.tbp * a.ldq);  // tile

    const int64_t g = a.tnodes[blockIdx.x];
    const int T = a.t_cnt[g];
    if (T == 0) return;
    const int64_t toff = a.t_off[g];
    const int64_t e0 = a.ptr[g], e1 = a.ptr[g + 1];
    const int ldq = a.ldq;
    const int tid = threadIdx.x;
    // targets per thread block row: T itself (at most a.tbp), so that no lane
    // of a group idles, but at least 16 lanes per group (at most 16 groups to
    // reduce); the remaining threads split the sources into groups
    const int tbp = min(max(T, (16 + a.nchunks - 1) / a.nchunks), a.tbp);
    const int groups = kKsThreads / (tbp * a.nchunks);
    const int per_group = tbp * a.nchunks;
    const int grp = tid / per_group;
    const int lt = tid % per_group;
    const int ta = lt % tbp;          // target within the block
    const int ch = lt / tbp;            // RHS chunk
    const bool active = grp < groups;

    for (int tb = 0; tb < T; tb += tbp) {
        const int tcount = min(tbp, T - tb);
        const bool have = active && ta < tcount;
        double xa = 0, ya = 0, za = 0;
        if (have) {
            P4 p = reinterpret_cast<const P4 *>(a.xt)[toff + tb + ta];
            xa = p.x; ya = p.y; za = p.z;
        }
        double acc[RC];
#pragma unroll
        for (int r = 0; r < RC; ++r) acc[r] = 0.0;
        // walk the source stream: partners e0..e1, each a run of points
        for (int64_t e = e0; e < e1;) {
            load_partner_chunk<kKsThreads>(pc, e, e1, a.col, a.s_off, a.s_cnt);
            const int nchunk = pc.n, total = pc.pre[pc.n];
            e += nchunk;
            for (int pos = 0; pos < total; pos += tile) {
            const int fill = min(tile, total - pos);
            for (int q = tid; q < fill; q += kKsThreads) sidx[q] = chunk_source(pc, pos + q);
            __syncthreads();
            for (int q = tid; q < fill; q += kKsThreads) sy[q] = reinterpret_cast<const P4 *>(a.ys)[sidx[q]];
            for (int q = tid; q < fill * ldq; q += kKsThreads) {
                int b = q / ldq, c = q % ldq;
                sq[q] = a.qv[sidx[b] * ldq + c];
            }
            __syncthreads();
            if (have) {
                for (int b = grp; b < fill; b += groups) {
                    P4 y = sy[b];
                    double kv = kappa64<KID>(xa - y.x, ya - y.y, za - y.z);
                    const double *qb = sq + (size_t)b * ldq + ch * RC;
                    if (RC >= 2) {
#pragma unroll
                        for (int r = 0; r < RC; r += 2) {
                            double2 v = *reinterpret_cast<const double2 *>(qb + r);
                            acc[r] += kv * v.x;
                            acc[r + 1] += kv * v.y;
                        }
                    } else {
                        acc[0] += kv * qb[0];
                    }
                }
            }
            __syncthreads();
            }
        }
        // deterministic reduction over the source groups
        for (int gg = 0; gg < groups; ++gg) {
            if (have && grp == gg) {
#pragma unroll
                for (int r = 0; r < RC; ++r) {
                    double *dst = red + (size_t)ta * ldq + ch * RC + r;
                    *dst = gg == 0 ? acc[r] : *dst + acc[r];
                }
            }
            __syncthreads();
        }
        for (int q = tid; q < tcount * ldq; q += kKsThreads) a.out[(toff + tb) * ldq + q] = red[q];
        __syncthreads();
    }
}

template <int KID>
static void launch_ksum(KsumArgs a, int64_t ntn, int RC, cudaStream_t s) {
    if (ntn <= 0) return;
    size_t smem = sizeof(P4) * a.tile + sizeof(double) * ((size_t)a.tile * a.ldq + (size_t)a.tbp * a.ldq) +
                  sizeof(int64_t) * a.tile;
    void (*kern)(KsumArgs) = nullptr;
    switch (RC) {
    case 1: kern = ksum_f64_kernel<KID, 1>; break;
    case 2: kern = ksum_f64_kernel<KID, 2>; break;
    case 4: kern = ksum_f64_kernel<KID, 4>; break;
    case 8: kern = ksum_f64_kernel<KID, 8>; break;
    case 16: kern = ksum_f64_kernel<KID, 16>; break;
    default: kern = ksum_f64_kernel<KID, 32>; break;
    }
    allow_max_dynamic_smem((const void *)kern);
    kern<<<(unsigned)ntn, kKsThreads, smem, s>>>(a);
    LAUNCHED();
}

static void ksum_launch(int kid, KsumArgs a, int64_t ntn, int RC, cudaStream_t s) {
    switch (kid) {
    case SMASH_K_LOG: launch_ksum<SMASH_K_LOG>(a, ntn, RC, s); break;
    case SMASH_K_INVR: launch_ksum<SMASH_K_INVR>(a, ntn, RC, s); break;
    case SMASH_K_YUKAWA: launch_ksum<SMASH_K_YUKAWA>(a, ntn, RC, s); break;
    case SMASH_K_DLP1: launch_ksum<SMASH_K_DLP1>(a, ntn, RC, s); break;
    case SMASH_K_DLP2: launch_ksum<SMASH_K_DLP2>(a, ntn, RC, s); break;
    default: launch_ksum<SMASH_K_CAUCHY1D>(a, ntn, RC, s); break;
    }
}

// Thread shape: tbp targets x nchunks RHS chunks x groups over sources.  With
// tuning (h != nullptr), bit 0 of the choice halves the source tile and bit 1
// halves the target block cap.
static void ksum(const smash_h2 *h, int kid, KsumArgs a, int64_t ntn, int max_targets, int RC, cudaStream_t s) {
    a.nchunks = a.ldq / RC;
    int tbp = 32;
    while (tbp < max_targets && tbp * 2 * a.nchunks <= kKsThreads) tbp *= 2;
    if (tbp * a.nchunks > kKsThreads) tbp = std::max(1, kKsThreads / a.nchunks);
    auto run = [&](int c) {
        KsumArgs b = a;
        b.tile = (c & 1) ? kKsTile / 2 : kKsTile;
        b.tbp = (c & 2) ? tbp / 2 : tbp;
        b.groups = std::max(1, kKsThreads / (b.tbp * b.nchunks));
        ksum_launch(kid, b, ntn, RC, s);
    };
    if (!h) {
        run(0);
        return;
    }
    std::vector<int> cands = {0, 1};
    if (tbp >= 64) { cands.push_back(2); cands.push_back(3); }
    char key[160];
    std::snprintf(key, sizeof(key), "ksum_f64/sm%d/k%d/rc%d/ld%d/t%lld/n%lld", h->num_sms, kid, RC, a.ldq,
                  pow2_at_least(max_targets), pow2_at_least(ntn));
    tune_choose(key, cands, 0, s, run);
}

// ------------------------------------------------------------------ driver
static void rhs_layout(int nrhs, int &ldq, int &RC) {
    if (nrhs <= 32) {
        RC = 1;
        while (RC < nrhs) RC *= 2;
        ldq = RC;
    } else {
        RC = 32;
        ldq = (nrhs + 31) / 32 * 32;
    }
}

void matvec_f64(const smash_h2 *h, const double *X, double *Y, int nrhs, cudaStream_t s, Profile *prof, int kid) {
    const Side &R = h->row;
    const Side &Cs = *h->col;
    int ldq, RC;
    rhs_layout(nrhs, ldq, RC);
    Arena tmp(s);
    double *qs = tmp.alloc<double>((size_t)h->ny * ldq);
    double *zs = tmp.alloc<double>((size_t)h->nx * ldq);
    double *qhat = tmp.alloc<double>((size_t)std::max<int64_t>(Cs.total_skel, 1) * ldq);
    double *zhat = tmp.alloc<double>((size_t)std::max<int64_t>(R.total_skel, 1) * ldq);
    PhaseTimer tm(s, prof);
    tm.mark();
    gather_rhs_kernel<<<(unsigned)((h->ny * ldq + 255) / 256), 256, 0, s>>>(X, nrhs, h->permy, h->ny, ldq, qs);
    LAUNCHED();
    tm.mark();
    // near field: every point belongs to one leaf, so zs is written in full
    {
        KsumArgs a{};
        a.tnodes = h->leaf_list; a.t_off = h->rs; a.t_cnt = h->rc;
        a.ptr = h->near_ptr; a.col = h->near_col; a.s_off = h->cs; a.s_cnt = h->cc;
        a.xt = h->xs; a.ys = h->ys; a.qv = qs; a.out = zs; a.ldq = ldq;
        ksum(h, kid, a, h->nleaves, std::min<int64_t>(h->leaf_size, 256), RC, s);
    }
    tm.mark();
    for (int l = h->L; l >= 2; --l) {
        int64_t n0 = h->lvl_off[l - 1], nl = h->lvl_off[l] - n0;
        PassArgs p{n0, h->leaf, Cs.m, Cs.k, Cs.in_off, Cs.sk_off, Cs.loc_off, Cs.g_off, Cs.loc, Cs.G,
                   qs, qhat, qhat, nullptr, ldq};
        upward_kernel<<<(unsigned)nl, 256, 0, s>>>(p);
        LAUNCHED();
    }
    tm.mark();
    if (h->nnodes > h->nroots) {
        KsumArgs a{};
        a.tnodes = h->nonroot_list; a.t_off = R.sk_off; a.t_cnt = R.k;
        a.ptr = h->adm_ptr; a.col = h->adm_col; a.s_off = Cs.sk_off; a.s_cnt = Cs.k;
        a.xt = R.skel_xyz; a.ys = Cs.skel_xyz; a.qv = qhat; a.out = zhat; a.ldq = ldq;
        ksum(h, kid, a, h->nnodes - h->nroots, h->r, RC, s);
    }
    tm.mark();
    for (int l = 2; l <= h->L; ++l) {
        int64_t n0 = h->lvl_off[l - 1], nl = h->lvl_off[l] - n0;
        PassArgs p{n0, h->leaf, R.m, R.k, R.in_off, R.sk_off, R.loc_off, R.g_off, R.loc, R.G,
                   nullptr, zhat, zhat, zs, ldq};
        downward_kernel<<<(unsigned)nl, 256, 0, s>>>(p);
        LAUNCHED();
    }
    tm.mark();
    scatter_rhs_kernel<<<(unsigned)((h->nx * nrhs + 255) / 256), 256, 0, s>>>(zs, ldq, h->permx, h->nx, nrhs, Y);
    LAUNCHED();
    tm.mark();
    tm.finish(4);
    tmp.release();
}

// ------------------------------------------------------------------ pass helpers
// The gather, transfer and scatter passes of matvec_f64 as separate calls,
// shared by the double-float matvec.
void matvec_gather(const smash_h2 *h, const double *X, int nrhs, int ldq, double *qs, cudaStream_t s) {
    gather_rhs_kernel<<<(unsigned)((h->ny * ldq + 255) / 256), 256, 0, s>>>(X, nrhs, h->permy, h->ny, ldq, qs);
    LAUNCHED();
}

void matvec_upward(const smash_h2 *h, const double *qs, double *qhat, int ldq, cudaStream_t s) {
    const Side &Cs = *h->col;
    for (int l = h->L; l >= 2; --l) {
        int64_t n0 = h->lvl_off[l - 1], nl = h->lvl_off[l] - n0;
        PassArgs p{n0, h->leaf, Cs.m, Cs.k, Cs.in_off, Cs.sk_off, Cs.loc_off, Cs.g_off, Cs.loc, Cs.G,
                   qs, qhat, qhat, nullptr, ldq};
        upward_kernel<<<(unsigned)nl, 256, 0, s>>>(p);
        LAUNCHED();
    }
}

void matvec_downward(const smash_h2 *h, double *zhat, double *zs, int ldq, cudaStream_t s) {
    const Side &R = h->row;
    for (int l = 2; l <= h->L; ++l) {
        int64_t n0 = h->lvl_off[l - 1], nl = h->lvl_off[l] - n0;
        PassArgs p{n0, h->leaf, R.m, R.k, R.in_off, R.sk_off, R.loc_off, R.g_off, R.loc, R.G,
                   nullptr, zhat, zhat, zs, ldq};
        downward_kernel<<<(unsigned)nl, 256, 0, s>>>(p);
        LAUNCHED();
    }
}

void matvec_scatter(const smash_h2 *h, const double *zs, int ldq, int nrhs, double *Y, cudaStream_t s) {
    scatter_rhs_kernel<<<(unsigned)((h->nx * nrhs + 255) / 256), 256, 0, s>>>(zs, ldq, h->permx, h->nx, nrhs, Y);
    LAUNCHED();
}

// ------------------------------------------------------------------ caller scratch
// The passes of matvec_f64 with qs, zs, q^ and z^ carved out of a caller
// buffer instead of stream-ordered allocations.  Every carved region is
// written in full before it is read (gather writes qs, the near field writes
// zs for every point, the upward pass writes every column skeleton slot, the
// coupling writes every row skeleton slot), so nothing needs clearing.
static size_t carve(size_t &off, size_t bytes) {
    size_t at = (off + 255) & ~size_t(255);
    off = at + bytes;
    return at;
}

size_t matvec_f64_scratch_bytes(const smash_h2 *h, int nrhs) {
    int ldq, RC;
    rhs_layout(nrhs, ldq, RC);
    size_t off = 0;
    carve(off, sizeof(double) * (size_t)h->ny * ldq);
    carve(off, sizeof(double) * (size_t)h->nx * ldq);
    carve(off, sizeof(double) * (size_t)std::max<int64_t>(h->col->total_skel, 1) * ldq);
    carve(off, sizeof(double) * (size_t)std::max<int64_t>(h->row.total_skel, 1) * ldq);
    return off;
}

void matvec_f64_scratch(const smash_h2 *h, const double *X, double *Y, int nrhs, cudaStream_t s, void *scratch,
                        size_t scratch_bytes) {
    const Side &R = h->row;
    const Side &Cs = *h->col;
    int ldq, RC;
    rhs_layout(nrhs, ldq, RC);
    if (matvec_f64_scratch_bytes(h, nrhs) > scratch_bytes) fail(SMASH_EINVAL, "scratch too small");
    unsigned char *base = static_cast<unsigned char *>(scratch);
    size_t off = 0;
    double *qs = reinterpret_cast<double *>(base + carve(off, sizeof(double) * (size_t)h->ny * ldq));
    double *zs = reinterpret_cast<double *>(base + carve(off, sizeof(double) * (size_t)h->nx * ldq));
    double *qhat = reinterpret_cast<double *>(
        base + carve(off, sizeof(double) * (size_t)std::max<int64_t>(Cs.total_skel, 1) * ldq));
    double *zhat = reinterpret_cast<double *>(
        base + carve(off, sizeof(double) * (size_t)std::max<int64_t>(R.total_skel, 1) * ldq));
    gather_rhs_kernel<<<(unsigned)((h->ny * ldq + 255) / 256), 256, 0, s>>>(X, nrhs, h->permy, h->ny, ldq, qs);
    LAUNCHED();
    {
        KsumArgs a{};
        a.tnodes = h->leaf_list; a.t_off = h->rs; a.t_cnt = h->rc;
        a.ptr = h->near_ptr; a.col = h->near_col; a.s_off = h->cs; a.s_cnt = h->cc;
        a.xt = h->xs; a.ys = h->ys; a.qv = qs; a.out = zs; a.ldq = ldq;
        // nullptr handle: the untuned default shape of each kernel sum, so that
        // this path never times candidates (tuning allocates); it can be slower
        // than the shape smash_matvec_ex picks with tuning on
        ksum(nullptr, h->kernel_id, a, h->nleaves, std::min<int64_t>(h->leaf_size, 256), RC, s);
    }
    for (int l = h->L; l >= 2; --l) {
        int64_t n0 = h->lvl_off[l - 1], nl = h->lvl_off[l] - n0;
        PassArgs p{n0, h->leaf, Cs.m, Cs.k, Cs.in_off, Cs.sk_off, Cs.loc_off, Cs.g_off, Cs.loc, Cs.G,
                   qs, qhat, qhat, nullptr, ldq};
        upward_kernel<<<(unsigned)nl, 256, 0, s>>>(p);
        LAUNCHED();
    }
    if (h->nnodes > h->nroots) {
        KsumArgs a{};
        a.tnodes = h->nonroot_list; a.t_off = R.sk_off; a.t_cnt = R.k;
        a.ptr = h->adm_ptr; a.col = h->adm_col; a.s_off = Cs.sk_off; a.s_cnt = Cs.k;
        a.xt = R.skel_xyz; a.ys = Cs.skel_xyz; a.qv = qhat; a.out = zhat; a.ldq = ldq;
        ksum(nullptr, h->kernel_id, a, h->nnodes - h->nroots, h->r, RC, s);
    }
    for (int l = 2; l <= h->L; ++l) {
        int64_t n0 = h->lvl_off[l - 1], nl = h->lvl_off[l] - n0;
        PassArgs p{n0, h->leaf, R.m, R.k, R.in_off, R.sk_off, R.loc_off, R.g_off, R.loc, R.G,
                   nullptr, zhat, zhat, zs, ldq};
        downward_kernel<<<(unsigned)nl, 256, 0, s>>>(p);
        LAUNCHED();
    }
    scatter_rhs_kernel<<<(unsigned)((h->nx * nrhs + 255) / 256), 256, 0, s>>>(zs, ldq, h->permx, h->nx, nrhs, Y);
    LAUNCHED();
}

}  // namespace smash
