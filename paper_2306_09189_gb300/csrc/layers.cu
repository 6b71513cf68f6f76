// The paper's layer programs on sharded ciphertexts (Sec. 4): the host planner (layout
// metadata, rotation sets, diagonal plaintexts, pooling masks) and the drivers that run the
// key switches, the fused plaintext x ciphertext MAC and the rescales on the device.
//
// Two execution modes give the same bits: HE_PLAIN launches the key-switching kernels one
// rotation at a time; HE_BATCHED raises every source once and puts every rotation of a stage
// into one launch per kernel (inner product, ModDown, NTTs), in chunks sized to memory.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <array>
#include <cmath>
#include <complex>
#include <functional>
#include <thread>
#include <unordered_map>
#include <set>
#include <tuple>

#include "internal.h"

namespace {

// ================================================================================ layout
struct Lay {
    int c = 0, m = 0, M = 0, N = 0, B = 0, ns = 0, nb = 0;
    std::vector<int> chan, row0;
    int rows() const { return B / M; }
};

Lay from_c(const he_layout &l) {
    Lay r;
    r.c = l.c; r.m = l.m; r.M = l.M; r.N = l.N; r.B = l.B; r.ns = l.n_shards; r.nb = l.nb;
    size_t cnt = (size_t)std::max(0, l.n_shards) * std::max(0, l.nb);
    cnt = std::min<size_t>(cnt, HE_MAX_BLOCKS);
    r.chan.assign(l.chan, l.chan + cnt);
    r.row0.assign(l.row0, l.row0 + cnt);
    return r;
}

int to_c(const Lay &r, he_layout *l) {
    if ((size_t)r.ns * r.nb > HE_MAX_BLOCKS) {
        he_set_error("layout needs %d blocks > HE_MAX_BLOCKS", r.ns * r.nb);
        return HE_EINVAL;
    }
    memset(l, 0, sizeof(*l));
    l->c = r.c; l->m = r.m; l->M = r.M; l->N = r.N; l->B = r.B; l->n_shards = r.ns; l->nb = r.nb;
    for (size_t i = 0; i < r.chan.size(); i++) {
        l->chan[i] = r.chan[i];
        l->row0[i] = r.row0[i];
    }
    return HE_OK;
}

int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

int check_layout(const Lay &l, int N) {
    bool ok = l.M > 0 && !(l.M & (l.M - 1)) && l.m >= 1 && l.m <= l.M && l.N == N && l.B > 0 &&
              l.N % l.B == 0 && l.B % l.M == 0 && l.nb == l.N / l.B && l.ns >= 1 && l.c >= 1 &&
              (size_t)l.ns * l.nb <= HE_MAX_BLOCKS;
    if (!ok) {
        he_set_error("inconsistent layout (frame, block or shard sizes)");
        return HE_EINVAL;
    }
    for (size_t i = 0; i < l.chan.size(); i++)
        if (l.chan[i] >= l.c || l.chan[i] < -1 || l.row0[i] < 0) {
            he_set_error("layout table out of range");
            return HE_EINVAL;
        }
    return HE_OK;
}

Lay image_layout(int c, int m, int N) {
    Lay L;
    L.c = c; L.m = m; L.M = next_pow2(m); L.N = N;
    const int M = L.M;
    if ((long long)M * M <= N) {
        L.B = M * M;
        L.nb = N / L.B;
        if ((long long)c * L.B <= N) {              // one shard, tiled duplication
            L.ns = 1;
            L.chan.assign(L.nb, -1);
            int d = L.nb / c;
            for (int b = 0; b < d * c; b++) L.chan[b] = b % c;
        } else {                                    // image shards
            L.ns = (c + L.nb - 1) / L.nb;
            L.chan.assign((size_t)L.ns * L.nb, -1);
            for (int f = 0; f < c; f++) L.chan[f] = f;
        }
        L.row0.assign(L.chan.size(), 0);
    } else {                                        // channel shards
        L.B = N;
        L.nb = 1;
        const int R = N / M, h = M / R;
        L.ns = c * h;
        L.chan.resize(L.ns);
        L.row0.resize(L.ns);
        for (int f = 0; f < c; f++)
            for (int k = 0; k < h; k++) {
                L.chan[f * h + k] = f;
                L.row0[f * h + k] = k * R;
            }
    }
    return L;
}

struct SlotInfo {
    int ch, y, x;
    bool valid;
};
inline SlotInfo slot_info(const Lay &L, int u, int i) {
    int b = i / L.B;
    SlotInfo s;
    s.ch = L.chan[(size_t)u * L.nb + b];
    s.y = L.row0[(size_t)u * L.nb + b] + (i % L.B) / L.M;
    s.x = i % L.M;
    s.valid = s.ch >= 0 && s.y < L.m && s.x < L.m;
    return s;
}

// ================================================================================ conv plan
// For output slot i of shard v (channel o, pixel (y, x)), input channel f and tap (k, l), the
// source pixel (y+k-pad, x+l-pad), when inside the image, is read from the copy of channel f
// holding that row; among duplicated copies the smallest block offset (b_in - b_out) mod nb
// wins, then the lowest shard.  Amount a = (j - i) mod N and D_{u,v,a}[i] = W[o][f][k][l]:
// Eq. 1 (shift with its binary mask merged into the weight), Eqs. 2-5 (rotation by
// r m^2 + shift), Eq. 6 (image shards), the tau/duplication indexing rule, Eq. 7 (channel
// shards: own and neighbour shard share one amount).
typedef std::map<long long, std::vector<double>> DiagMap;   // key u*N + a, ascending

void plan_conv_v(const Lay &lin, const Lay &lout, const double *W, int ci, int kh, int kw,
                 int pad, int v, DiagMap &out) {
    const int N = lin.N;
    struct Copy { int u, b, r0; };
    std::vector<std::vector<Copy>> copies(ci);
    for (int u = 0; u < lin.ns; u++)
        for (int b = 0; b < lin.nb; b++) {
            int f = lin.chan[(size_t)u * lin.nb + b];
            if (f >= 0) copies[f].push_back({u, b, lin.row0[(size_t)u * lin.nb + b]});
        }
    const int R = lin.rows();
    for (int i = 0; i < N; i++) {
        SlotInfo so = slot_info(lout, v, i);
        if (!so.valid) continue;
        const int b_out = i / lout.B;
        for (int f = 0; f < ci; f++)
            for (int k = 0; k < kh; k++) {
                const int ys = so.y + k - pad;
                if (ys < 0 || ys >= lin.m) continue;
                for (int l = 0; l < kw; l++) {
                    const int xs = so.x + l - pad;
                    if (xs < 0 || xs >= lin.m) continue;
                    long long bestkey = -1, j = 0;
                    int bu = -1;
                    for (const Copy &cp : copies[f]) {
                        if (ys < cp.r0 || ys >= cp.r0 + R) continue;
                        long long key = (long long)(((cp.b - b_out) % lin.nb + lin.nb) % lin.nb) * (lin.ns + 1) + cp.u;
                        if (bu < 0 || key < bestkey) {
                            bestkey = key;
                            j = (long long)cp.b * lin.B + (long long)(ys - cp.r0) * lin.M + xs;
                            bu = cp.u;
                        }
                    }
                    if (bu < 0) continue;
                    const int a = (int)(((j - i) % N + N) % N);
                    std::vector<double> &D = out[(long long)bu * N + a];
                    if (D.empty()) D.assign(N, 0.0);
                    D[i] = W[(((size_t)so.ch * ci + f) * kh + k) * kw + l];
                }
            }
    }
}

// ================================================================================ pool plan
// Sec. 4.2.  S: W = X + rot_1 X + rot_M X + rot_{M+1} X (2x2 ones convolution; skipped for the
// stride-2 select).  H (Eq. 10): Y = sum_{x'} mask_{x'} rot_{x'}(W) on even valid rows, column
// x'.  V (Eq. 11): Z = sum_{y'} mask_{y'} rot_{3 y' M / 2}(Y).  C (Eq. 12): shard 4g+q's old
// block b becomes block 4b+q of output shard g (rotation right by q B/4).  Duplication
// (Eq. 13) when 1 or 2 shards remain.
struct PoolPlanH {
    Lay lin, lout;
    std::vector<int> pre, h_amt, v_amt;
    std::vector<std::vector<std::vector<double>>> h_mask, v_mask;    // [amount][shard][N]
    std::vector<std::vector<std::pair<int, int>>> groups;             // [out][(in shard, amount)]
    std::vector<int> dup;                                             // incl. 0
};

int plan_pool(const Lay &lin, bool select, PoolPlanH &P) {
    const int M = lin.M, N = lin.N, B = lin.B, m = lin.m;
    if (m % 2 || M < 2 || lin.rows() % 2) {
        he_set_error("pooling needs an even image side and an even number of rows per block");
        return HE_EINVAL;
    }
    P.lin = lin;
    const double w = select ? 1.0 : 0.25;
    if (!select) P.pre = {0, 1, M, M + 1};
    const int Mh = M / 2, Rb = lin.rows();
    for (int xp = 0; xp < m / 2; xp++) {
        std::vector<std::vector<double>> mk(lin.ns, std::vector<double>(N, 0.0));
        for (int u = 0; u < lin.ns; u++)
            for (int i = xp; i < N; i += M) {
                int blk = i / B;
                int ch = lin.chan[(size_t)u * lin.nb + blk];
                int y = lin.row0[(size_t)u * lin.nb + blk] + (i % B) / M;
                if (ch >= 0 && y % 2 == 0 && y < m) mk[u][i] = w;
            }
        P.h_amt.push_back(xp);
        P.h_mask.push_back(std::move(mk));
    }
    for (int yp = 0; yp < Rb / 2; yp++) {
        std::vector<std::vector<double>> mk(lin.ns, std::vector<double>(N, 0.0));
        bool any = false;
        for (int u = 0; u < lin.ns; u++)
            for (int i = 0; i < N; i++) {
                int blk = i / B, loc = i % B;
                int ch = lin.chan[(size_t)u * lin.nb + blk];
                int ynew = lin.row0[(size_t)u * lin.nb + blk] / 2 + yp;
                if (ch >= 0 && loc >= yp * Mh && loc < yp * Mh + m / 2 && ynew < m / 2) {
                    mk[u][i] = 1.0;
                    any = true;
                }
            }
        if (any) {
            P.v_amt.push_back(3 * yp * M / 2);
            P.v_mask.push_back(std::move(mk));
        }
    }
    const int Bn = B / 4, nbn = N / Bn, t = lin.ns, nout = (t + 3) / 4;
    Lay lo;
    lo.c = lin.c; lo.m = m / 2; lo.M = Mh; lo.N = N; lo.B = Bn; lo.ns = nout; lo.nb = nbn;
    lo.chan.assign((size_t)nout * nbn, -1);
    lo.row0.assign((size_t)nout * nbn, 0);
    for (int g = 0; g < nout; g++) {
        std::vector<std::pair<int, int>> grp;
        for (int q = 0; q < 4; q++) {
            int s = 4 * g + q;
            if (s >= t) break;
            grp.push_back({s, ((-q * Bn) % N + N) % N});
            for (int b = 0; b < lin.nb; b++) {
                lo.chan[(size_t)g * nbn + 4 * b + q] = lin.chan[(size_t)s * lin.nb + b];
                lo.row0[(size_t)g * nbn + 4 * b + q] = lin.row0[(size_t)s * lin.nb + b] / 2;
            }
        }
        P.groups.push_back(grp);
    }
    P.dup = {0};
    if (t == 1 || t == 2) {
        const int f = 4 / t, step = t * Bn;
        P.dup.clear();
        for (int k = 0; k < f; k++) P.dup.push_back(((-k * step) % N + N) % N);
        // block b of the duplicated shard is the sum of the consolidated blocks b - k t (k < f):
        // its channel is the one of those consolidated blocks that holds data, so read the
        // table as it was before duplication (an empty block stays empty)
        const std::vector<int> chan0 = lo.chan, row00 = lo.row0;
        for (int k = 1; k < f; k++)
            for (int b = 0; b < nbn; b++) {
                int src = b - k * (step / Bn);
                if (src >= 0 && chan0[src] >= 0 && lo.chan[b] < 0) {
                    lo.chan[b] = chan0[src];
                    lo.row0[b] = row00[src];
                }
            }
    }
    P.lout = lo;
    return HE_OK;
}

// ================================================================================ helpers
template <class T>
int dev_alloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) return HE_OK;
    HE_TRY(he_capture_guard("device allocation"));
    if (he_alloc_should_fail() || he_malloc((void **)p, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        he_set_error("device allocation of %zu bytes failed", count * sizeof(T));
        return HE_ENOMEM;
    }
    return HE_OK;
}

he_ct view(he_ctx *c, u64 *d, size_t ps, int level, double scale) {
    he_ct t;
    t.ctx = c; t.d = d; t.pstride = ps; t.level = level; t.cap = level; t.scale = scale; t.owned = false;
    return t;
}

// Encode slot vectors at scale S (or take given integer plaintexts) and store them as
// Montgomery NTT-form plaintexts at `level`, contiguous [count][level+1][n] from dst.
int upload_plaintexts(he_ctx *c, const std::vector<const double *> &vecs, size_t count, double S,
                      int level, u64 *dst, const int64_t *given, bool ext = false) {
    const int n = c->n;
    const int nl = level + 1 + (ext ? c->K : 0);         // limbs stored: Q_l, or Q_l u P
    const size_t pw = (size_t)nl * n;
    int64_t *stage = (int64_t *)c->sc_tmp.p;
    const size_t cap = std::max<size_t>(1, std::min<size_t>(64, c->sc_tmp.words / n));
    std::vector<int64_t> host(cap * (size_t)n);
    for (size_t b0 = 0; b0 < count; b0 += cap) {
        const size_t nb = std::min(cap, count - b0);
        if (given) {
            memcpy(host.data(), given + b0 * n, nb * n * 8);
        } else {
            const unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
            std::vector<std::thread> th;
            for (unsigned t = 0; t < nt; t++)
                th.emplace_back([&, t]() {
                    for (size_t i = t; i < nb; i += nt) encode_slots(vecs[b0 + i], n, S, host.data() + i * n);
                });
            for (auto &x : th) x.join();
        }
        HE_CHECK_CUDA(cudaMemcpy(stage, host.data(), nb * n * 8, cudaMemcpyHostToDevice));
        for (size_t i = 0; i < nb; i++)
            HE_TRY(k_reduce_int(c, stage + i * n, dst + (b0 + i) * pw, nl, level + 1, false, 0));
        ntt_job j{dst + b0 * pw, pw, 0, nl, level + 1, 0, (int)nb};
        HE_TRY(k_ntt(c, j, false, 0));
        HE_TRY(k_to_mont(c, dst + b0 * pw, nl, level + 1, (int)nb, pw, 0));
        HE_CHECK_CUDA(cudaStreamSynchronize(0));
    }
    return HE_OK;
}

// normal-form NTT addend at `level` from an integer polynomial
int upload_addend(he_ctx *c, const int64_t *m, int level, u64 *dst) {
    int64_t *stage = (int64_t *)c->sc_tmp.p;
    HE_CHECK_CUDA(cudaMemcpy(stage, m, (size_t)c->n * 8, cudaMemcpyHostToDevice));
    HE_TRY(k_reduce_int(c, stage, dst, level + 1, level + 1, false, 0));
    ntt_job j{dst, 0, 0, level + 1, level + 1, 0, 1};
    HE_TRY(k_ntt(c, j, false, 0));
    HE_CHECK_CUDA(cudaStreamSynchronize(0));
    return HE_OK;
}

size_t autotune_chunk(he_ctx *c, int level, size_t items) {
    // one chunk's inner-product outputs and ModDown buffers stay under 4 GiB
    size_t per = (size_t)(2 * (level + 1 + c->K) + 2 * (level + 1)) * c->n * 8;
    size_t cap = std::max<size_t>(1, ((size_t)4 << 30) / per);
    return std::max<size_t>(1, std::min(cap, items));
}

}  // namespace

// ================================================================================ rotation sets
// Hoisted rotations of several sources (ModUp of c1 once per source, Sec. 4.1 "computed once
// and cached"), each by its own amounts, into destination buffers.
struct RotSet {
    he_ctx *c = nullptr;
    int level = 0;
    struct Src { u64 *d; size_t ps; };
    struct Item { int src, amount; u64 g; u64 *dst; size_t ps; };
    std::vector<Src> src;
    std::vector<Item> items;                                   // non-zero amounts, by source
    struct Copy { int src; u64 *dst; size_t ps; };
    std::vector<Copy> copies;                                  // amount 0
    std::vector<const DeviceKey *> keys;
    size_t chunk = 0;
    u64 *D_all = nullptr, *u_all = nullptr, *conv_all = nullptr;
    u64 *htmp = nullptr;                                       // [src][nq][n] gathered c1
    modup_src *d_hsrc = nullptr;
    ip_item *d_ip = nullptr;
    md_item *d_md = nullptr;
    bool batched_ready = false;

    ~RotSet() {
        he_free(D_all); he_free(u_all); he_free(conv_all); he_free(d_ip); he_free(d_md);
        he_free(htmp); he_free(d_hsrc);
    }
    size_t nq() const { return (size_t)level + 1; }
    size_t pw() const { return nq() * c->n; }
    size_t ext() const { return (nq() + c->K) * c->n; }
    int beta() const { return (level + c->alpha) / c->alpha; }

    void add(int s, int amount, u64 *dst, size_t ps) {
        u64 g = h_galois(c, amount);
        if (g == 1) copies.push_back({s, dst, ps});
        else items.push_back({s, amount, g, dst, ps});
    }

    int resolve_keys() {
        keys.resize(items.size());
        for (size_t i = 0; i < items.size(); i++) HE_TRY(get_key(c, (int)items[i].g, &keys[i]));
        return HE_OK;
    }

    int prepare_batched() {
        HE_TRY(resolve_keys());
        if (batched_ready || items.empty()) { batched_ready = true; return HE_OK; }
        chunk = autotune_chunk(c, level, items.size());
        HE_TRY(dev_alloc(&D_all, src.size() * (size_t)beta() * ext()));
        HE_TRY(dev_alloc(&htmp, src.size() * pw()));
        {
            std::vector<modup_src> hs(src.size());
            for (size_t u = 0; u < src.size(); u++) hs[u] = modup_src{src[u].d + src[u].ps, D_all + u * (size_t)beta() * ext()};
            HE_TRY(dev_alloc(&d_hsrc, hs.size()));
            HE_CHECK_CUDA(cudaMemcpy(d_hsrc, hs.data(), hs.size() * sizeof(modup_src), cudaMemcpyHostToDevice));
        }
        HE_TRY(dev_alloc(&u_all, chunk * 2 * ext()));
        HE_TRY(dev_alloc(&conv_all, chunk * 2 * pw()));
        std::vector<ip_item> ip(items.size());
        std::vector<md_item> md(items.size());
        for (size_t i = 0; i < items.size(); i++) {
            const Item &it = items[i];
            const size_t slot = i % chunk;
            ip[i] = ip_item{D_all + (size_t)it.src * beta() * ext(), keys[i]->d,
                            u_all + slot * 2 * ext(), it.g, beta()};
            md[i] = md_item{u_all + slot * 2 * ext(), conv_all + slot * 2 * pw(), src[it.src].d,
                            src[it.src].ps, 1, it.g, it.dst, it.ps};
        }
        HE_TRY(dev_alloc(&d_ip, ip.size()));
        HE_TRY(dev_alloc(&d_md, md.size()));
        HE_CHECK_CUDA(cudaMemcpy(d_ip, ip.data(), ip.size() * sizeof(ip_item), cudaMemcpyHostToDevice));
        HE_CHECK_CUDA(cudaMemcpy(d_md, md.data(), md.size() * sizeof(md_item), cudaMemcpyHostToDevice));
        batched_ready = true;
        return HE_OK;
    }

    int run(int mode, cudaStream_t s) {
        for (const Copy &cp : copies)
            HE_TRY(k_copy_limbs(cp.dst, cp.ps, src[cp.src].d, src[cp.src].ps, pw(), 2, s));
        if (items.empty()) return HE_OK;
        if (keys.size() != items.size()) HE_TRY(resolve_keys());
        if (mode == HE_PLAIN) {
            int cur = -1;
            for (size_t i = 0; i < items.size(); i++) {
                const Item &it = items[i];
                if (it.src != cur) {
                    he_ct t = view(c, src[it.src].d, src[it.src].ps, level, 1.0);
                    HE_TRY(hoist_modup(c, &t, c->sc_digits.p, s));
                    cur = it.src;
                }
                HE_TRY(ks_tail(c, c->sc_digits.p, level, *keys[i], it.g, src[it.src].d, src[it.src].ps,
                               1, it.g, it.dst, it.ps, s));
            }
            return HE_OK;
        }
        if (!batched_ready) HE_TRY(prepare_batched());
        // every source's ModUp in one launch set
        HE_TRY(k_modup_batch(c, d_hsrc, (int)src.size(), htmp, level, s));
        {
            ntt_job jd{D_all, ext(), 0, (int)nq() + c->K, (int)nq(), c->alpha, beta() * (int)src.size(), beta()};
            HE_TRY(k_ntt(c, jd, false, s));
        }
        const int nqi = (int)nq();
        for (size_t i0 = 0; i0 < items.size(); i0 += chunk) {
            const int cnt = (int)std::min(chunk, items.size() - i0);
            HE_TRY(k_inner_product(c, d_ip + i0, cnt, level, s));
            ntt_job jp{u_all, ext(), nqi, c->K, nqi, 0, 2 * cnt};
            HE_TRY(k_ntt(c, jp, true, s));
            HE_TRY(k_moddown_fbc(c, u_all, conv_all, level, 2 * cnt, s));
            ntt_job jc{conv_all, pw(), 0, nqi, nqi, 0, 2 * cnt};
            HE_TRY(k_ntt(c, jc, false, s));
            HE_TRY(k_moddown_combine(c, d_md + i0, cnt, level, s));
        }
        return HE_OK;
    }
};

// ================================================================================ fused stages
// One stage of weighted hoisted rotations: out_v = sum_{(s, a)} pt_{v,s,a} (.) rot_a(src_s),
// evaluated in the raised basis: every rotation's inner product is accumulated with its
// plaintext over Q u P (keys read once per amount and output group) and each output takes one
// ModDown.  Outputs are left unrescaled at the stage level.  A stage's groups (V outputs
// each) go into a FusedLaunch, which may also carry the groups of other stages (other images,
// other levels) so that all of them are served by one kernel launch.
struct FusedLaunch;

struct FusedStage {
    he_ctx *c = nullptr;
    int level = 0;
    int pt_level = -1;                                // layout of the plaintexts (default: level)
    struct Src { u64 *d; size_t ps; bool rotated; };
    std::vector<Src> srcs;
    struct Term { int v, s, a; const u64 *pt; };
    std::vector<Term> terms;
    std::vector<std::pair<u64 *, size_t>> outs;      // output data and poly stride
    struct Group {
        std::vector<int> outs;
        famt *d_amt = nullptr;
        fent *d_ent = nullptr;
        fgrp desc{};
        double bytes = 0, mulmods = 0;
    };
    std::vector<Group> groups;                        // for outputs-per-key-pass Vg
    std::vector<int> hslot;                           // source -> slot in D_all (-1: not rotated)
    int nh = 0;                                       // rotated sources
    u64 *D_all = nullptr;
    u64 *htmp = nullptr;                              // [nh][nq][n] c1 of the rotated sources
    modup_src *d_hsrc = nullptr;                      // [nh] their c1 and digit slots
    u64 *facc = nullptr, *fconv = nullptr;            // [nout][2][ext|nq][n]
    md_item *d_md = nullptr;
    bool ready = false;
    int Vg = 0;
    std::string name = "stage";
    std::unique_ptr<FusedLaunch> own;                 // launch of this stage alone
    // split form: chunks of keyed amounts (inner products into U, then the raised MAC)
    struct Chunk {
        famt *d_amt = nullptr;
        uent *d_ent = nullptr;
        ugrp udesc{};
        std::vector<rterm *> d_terms;                 // per output group of HE_RV
        std::vector<rgrp> rdesc;
        double ubytes = 0, rbytes = 0, rmm = 0;
        std::vector<std::pair<std::pair<int, int>, u64 *>> ukeys;   // (amount, source) -> U, ordered
    };
    std::vector<Chunk> chunks;
    u64 *U = nullptr;                                 // [slots][2][ext][n] of the largest chunk
    bool split_ready = false;
    // pre-keyed form (ipmac_pk_kernel): one group per output; per (output, keyed amount) with a
    // plaintext K' = key (.) pt in the key layout, per (output, amount) with a plaintext P pt
    struct PkGroup { famt *d_amt = nullptr; fent *d_ent = nullptr; fgrp desc{}; double bytes = 0, mulmods = 0; };
    std::vector<PkGroup> pk_groups;
    std::vector<std::array<uintptr_t, 4>> pk_refs;   // entries of the root's pre-keyed cache held
    bool pk_built = false;
    int pk_state = 0;                                 // 0: not checked, 1: eligible, -1: not
    uint64_t pk_epoch = 0;                            // bumped when the plaintexts are re-imported

    ~FusedStage();
    void free_pk() {
        for (auto &g : pk_groups) { he_free(g.d_amt); he_free(g.d_ent); }
        if (!pk_refs.empty()) {
            he_ctx *r = c->root();
            std::lock_guard<std::mutex> lk(r->pk_mu);
            for (auto &key : pk_refs) {
                auto it = r->pk_cache.find(key);
                if (it != r->pk_cache.end() && --it->second.refs == 0) {
                    he_free(it->second.Kp);
                    he_free(it->second.Ppt);
                    r->pk_cache.erase(it);
                }
            }
        }
        pk_groups.clear();
        pk_refs.clear();
        pk_built = false;
    }
    std::array<uintptr_t, 4> pk_key(const u64 *key, const u64 *pt) const {
        return {(uintptr_t)key, (uintptr_t)pt, (uintptr_t)level * 4096 + (uintptr_t)pt_level, (uintptr_t)pk_epoch};
    }
    void invalidate_pk();                             // plaintext contents changed
    // every output takes at most one source per amount
    bool pk_eligible() {
        if (pk_state == 0) {
            std::set<std::pair<int, int>> seen;
            pk_state = beta() <= 8 ? 1 : -1;
            for (auto &t : terms)
                if (!seen.insert({t.v, t.a}).second) { pk_state = -1; break; }
        }
        return pk_state > 0;
    }
    size_t pk_bytes() const {                         // new device memory the pre-keyed tables need
        const size_t kst = (size_t)(c->L + 1 + c->K) * c->n;
        size_t b = 0;
        he_ctx *r = c->root();
        std::lock_guard<std::mutex> lk(r->pk_mu);
        std::set<std::array<uintptr_t, 4>> fresh;     // distinct (key, plaintext) pairs to build
        for (auto &t : terms)
            if (t.pt && t.pt != HE_PT_ONE) {
                const u64 g = h_galois(c, t.a);
                auto kit = r->keys.find((int)g);
                const u64 *kd = (g != 1 && kit != r->keys.end()) ? kit->second.d : nullptr;
                const auto ck = pk_key(kd, t.pt);
                if (r->pk_cache.count(ck) || !fresh.insert(ck).second) continue;
                b += (size_t)nq() * c->n * 8;
                if (g != 1) b += (size_t)2 * beta() * kst * 8;
            }
        return b;
    }
    int build_pk();
    void free_split() {
        for (auto &ch : chunks) {
            he_free(ch.d_amt); he_free(ch.d_ent);
            for (auto *t : ch.d_terms) he_free(t);
        }
        chunks.clear();
        he_free(U);
        U = nullptr;
        split_ready = false;
    }
    size_t split_bytes() const;                       // device memory the split form needs
    int build_split(size_t cap_bytes, size_t plan_slot_bytes = 0);
    void free_groups() {
        for (auto &g : groups) { he_free(g.d_amt); he_free(g.d_ent); }
        groups.clear();
        Vg = 0;
    }
    int add_src(u64 *d, size_t ps) { srcs.push_back({d, ps, false}); return (int)srcs.size() - 1; }
    int add_out(u64 *d, size_t ps) { outs.push_back({d, ps}); return (int)outs.size() - 1; }
    void add_term(int v, int s, int a, const u64 *pt) { terms.push_back({v, s, ((a % c->N) + c->N) % c->N, pt}); }
    int nq() const { return level + 1; }
    int ext() const { return level + 1 + c->K; }
    int beta() const { return (level + c->alpha) / c->alpha; }

    int build() {
        if (ready) return HE_OK;
        if (pt_level < 0) pt_level = level;
        if (pt_level < level || pt_level > c->L) { he_set_error("fused stage: plaintext level below the stage"); return HE_EINVAL; }
        const size_t n = c->n, nout = outs.size();
        for (auto &t : terms)
            if (h_galois(c, t.a) != 1) srcs[t.s].rotated = true;
        hslot.assign(srcs.size(), -1);
        nh = 0;
        for (size_t i = 0; i < srcs.size(); i++)
            if (srcs[i].rotated) hslot[i] = nh++;
        HE_TRY(dev_alloc(&D_all, (size_t)nh * beta() * ext() * n));
        if (nh > 0) {
            HE_TRY(dev_alloc(&htmp, (size_t)nh * nq() * n));
            std::vector<modup_src> hs(nh);
            for (size_t i = 0; i < srcs.size(); i++)
                if (hslot[i] >= 0)
                    hs[hslot[i]] = modup_src{srcs[i].d + srcs[i].ps, D_all + (size_t)hslot[i] * beta() * ext() * n};
            HE_TRY(dev_alloc(&d_hsrc, hs.size()));
            HE_CHECK_CUDA(cudaMemcpy(d_hsrc, hs.data(), hs.size() * sizeof(modup_src), cudaMemcpyHostToDevice));
        }
        // a group stores only the outputs it has (fgrp.nv, rgrp.nv): no padding needed
        const size_t nslot = nout;
        HE_TRY(dev_alloc(&facc, nslot * 2 * ext() * n));
        HE_TRY(dev_alloc(&fconv, nslot * 2 * nq() * n));
        // the unrotated parts are folded into the raised sums, so the ModDown adds no base
        std::vector<md_item> md;
        for (size_t v = 0; v < nout; v++)
            md.push_back(md_item{facc + v * 2 * ext() * n, fconv + v * 2 * nq() * n, nullptr, 0, 0, 1,
                                 outs[v].first, outs[v].second});
        HE_TRY(dev_alloc(&d_md, std::max<size_t>(1, md.size())));
        if (!md.empty()) HE_CHECK_CUDA(cudaMemcpy(d_md, md.data(), md.size() * sizeof(md_item), cudaMemcpyHostToDevice));
        ready = true;
        return HE_OK;
    }

    // Groups of V outputs, each one group of the fused kernel: every key is streamed once for
    // the group's V outputs (and, through L2, for the neighbouring groups of the same launch).
    int build_groups(int V) {
        HE_TRY(build());
        if (V == Vg && !groups.empty()) return HE_OK;
        free_groups();
        Vg = V;
        const int nq_ = nq(), ext_ = ext(), beta_ = beta();
        const size_t n = c->n;
        std::vector<const u64 *> Dp(srcs.size());
        for (size_t i = 0; i < srcs.size(); i++)
            Dp[i] = hslot[i] >= 0 ? D_all + (size_t)hslot[i] * beta_ * ext_ * n : nullptr;
        const int nout = (int)outs.size();
        for (int v0 = 0; v0 < nout; v0 += V) {
            Group G;
            for (int v = v0; v < std::min(nout, v0 + V); v++) G.outs.push_back(v);
            // amount -> source -> per-output plaintexts
            std::map<int, std::map<int, fent>> m;
            for (auto &t : terms) {
                if (t.v < v0 || t.v >= v0 + V) continue;
                const int vi = t.v - v0;
                fent &e = m[t.a][t.s];
                e.s = t.s;
                if (e.pt[vi]) { he_set_error("fused stage: duplicate term"); return HE_EINVAL; }
                e.pt[vi] = t.pt;
            }
            std::vector<famt> ha;
            std::vector<fent> he;
            double bytes = 0, mm = 0;
            for (auto &am : m) {
                famt A;
                A.g = h_galois(c, am.first);
                A.key = nullptr;
                if (A.g != 1) {
                    const DeviceKey *k;
                    HE_TRY(get_key(c, (int)A.g, &k));
                    A.key = k->d;
                    bytes += (double)2 * beta_ * ext_ * n * 8;
                }
                A.e0 = (int)he.size();
                for (auto &se : am.second) {
                    fent E = se.second;
                    E.D = Dp[E.s];
                    E.src = srcs[E.s].d;
                    E.ps = srcs[E.s].ps;
                    he.push_back(E);
                    for (int vi = 0; vi < V; vi++)
                        if (se.second.pt[vi] && se.second.pt[vi] != HE_PT_ONE) bytes += (double)(A.key ? ext_ : nq_) * n * 8;
                    mm += (double)(A.key ? ext_ : nq_) * n * (A.key ? 2 * beta_ + 2 * V : 2 * V);
                }
                A.e1 = (int)he.size();
                ha.push_back(A);
            }
            bytes += (double)nh * beta_ * ext_ * n * 8 / std::max(1, (nout + V - 1) / V) +
                     (double)srcs.size() * 2 * nq_ * n * 8 / std::max(1, (nout + V - 1) / V) +
                     (double)G.outs.size() * 2 * ext_ * n * 8;
            G.bytes = bytes;
            G.mulmods = mm;
            HE_TRY(dev_alloc(&G.d_amt, std::max<size_t>(1, ha.size())));
            HE_TRY(dev_alloc(&G.d_ent, std::max<size_t>(1, he.size())));
            if (!ha.empty()) HE_CHECK_CUDA(cudaMemcpy(G.d_amt, ha.data(), ha.size() * sizeof(famt), cudaMemcpyHostToDevice));
            if (!he.empty()) HE_CHECK_CUDA(cudaMemcpy(G.d_ent, he.data(), he.size() * sizeof(fent), cudaMemcpyHostToDevice));
            G.desc = fgrp{G.d_amt, G.d_ent, (int)ha.size(), level, beta_, pt_level, (int)G.outs.size(),
                          facc + (size_t)v0 * 2 * ext_ * n};
            groups.push_back(G);
        }
        return HE_OK;
    }

    // ModUp of every rotated source: one gather, one INTT, one base conversion and one NTT
    // launch set for all of them (the bits of a ModUp per source)
    int hoist(cudaStream_t s) {
        if (nh == 0) return HE_OK;
        HE_TRY(k_modup_batch(c, d_hsrc, nh, htmp, level, s));
        ntt_job j{D_all, (size_t)ext() * c->n, 0, ext(), nq(), c->alpha, beta() * nh, beta()};
        return k_ntt(c, j, false, s);
    }

    // one ModDown pipeline for every output of the stage
    int moddown(cudaStream_t s) {
        const int nv = (int)outs.size();
        if (nv == 0) return HE_OK;
        ntt_job jp{facc, (size_t)ext() * c->n, nq(), c->K, nq(), 0, 2 * nv, 0};
        HE_TRY(k_ntt(c, jp, true, s));
        HE_TRY(k_moddown_fbc(c, facc, fconv, level, 2 * nv, s));
        ntt_job jc{fconv, (size_t)nq() * c->n, 0, nq(), nq(), 0, 2 * nv, 0};
        HE_TRY(k_ntt(c, jc, false, s));
        return k_moddown_combine(c, d_md, nv, level, s);
    }

    int run(cudaStream_t s);
};

// One fused-kernel launch over the groups of one or more stages.  Autotuner: the candidates
// (outputs per key pass V, key stream) give the same bits, so the first run times each one's
// launch (one warm-up pass, then the best of two timed passes, CUDA events on the launch's
// stream) and keeps the fastest.  Needs the raised digits in place: called after the hoisted
// ModUps of the first run.
static bool is_pk(int fm) {
    return fm == HE_KEY_STREAM_PK || fm == HE_KEY_STREAM_PK3 || fm == HE_KEY_STREAM_PKP || fm == HE_KEY_STREAM_PK1 ||
           fm == HE_KEY_STREAM_PKT || fm == HE_KEY_STREAM_PK3L;
}
static const char *pk_name(int fm) {
    return fm == HE_FORM_PK3 ? "pk3" : fm == HE_FORM_PKP ? "pkp" : fm == HE_KEY_STREAM_PK1 ? "pk1"
         : fm == HE_KEY_STREAM_PKT ? "pkt" : fm == HE_KEY_STREAM_PK3L ? "pk3l" : "pk";
}
static const char *form_name(int fm) {
    return fm == HE_KEY_STREAM_TMA ? "tma" : fm == HE_KEY_STREAM_CP ? "cp" : fm == HE_KEY_STREAM_LDG1 ? "ldg1" : "ldg";
}

struct FusedLaunch {
    he_ctx *c = nullptr;
    std::vector<FusedStage *> st;
    fgrp *d_grps = nullptr;
    int G = 0, V = 0, max_beta = 0;
    int gb = 0;                                       // groups per batch of the block schedule (0: all)
    int form = HE_KEY_STREAM_LDG;
    bool tuned = false;
    bool use_split = false;                           // split form chosen by the autotuner
    double bytes = 0, mulmods = 0;
    std::string name;
    // split form: per amount chunk, the inner-product and raised-MAC group tables
    std::vector<ugrp *> d_ugrps;
    std::vector<rgrp *> d_rgrps;
    std::vector<int> n_ugrp, n_rgrp;
    std::vector<double> ubytes, rbytes, rmm;
    bool split_built = false;
    // image-batched split form: per amount chunk, groups of HE_RNI stages x HE_RVM outputs
    std::vector<rgrp_m *> d_mgrps;
    std::vector<std::vector<rterm_m *>> d_mterms;
    std::vector<int> n_mgrp;
    std::vector<double> mbytes, mmm;
    bool splitm_built = false, use_split_m = false;
    // pre-keyed form: one group per output of every stage
    fgrp *d_pk = nullptr;
    int G_pk = 0;
    double pk_b = 0, pk_mm = 0;
    bool use_pk = false;

    ~FusedLaunch() { he_free(d_grps); he_free(d_pk); free_split_tables(); }
    // the stages of a batch share one plan (the same terms, sources and outputs; plaintexts and
    // their level): the image-batched split form applies
    bool splitm_ok() const {
        if (st.size() < 2) return false;
        const FusedStage *a = st[0];
        for (auto *f : st) {
            if (f->terms.size() != a->terms.size() || f->outs.size() != a->outs.size() ||
                f->srcs.size() != a->srcs.size() || f->pt_level != a->pt_level)
                return false;
            for (size_t i = 0; i < f->terms.size(); i++)
                if (f->terms[i].v != a->terms[i].v || f->terms[i].s != a->terms[i].s || f->terms[i].a != a->terms[i].a ||
                    f->terms[i].pt != a->terms[i].pt)
                    return false;
        }
        return true;
    }
    int build_split_m() {
        if (splitm_built) return HE_OK;
        HE_TRY(build_split());
        const size_t nch = st[0]->chunks.size();
        for (auto *f : st)
            if (f->chunks.size() != nch) { he_set_error("image-batched split: chunk plans differ"); return HE_ESTATE; }
        const FusedStage *a = st[0];
        const int nout = (int)a->outs.size();
        std::map<std::array<int, 3>, const u64 *> ptm;            // (amount, source, output) -> plaintext
        for (auto &t : a->terms) ptm[{h_galois(c, t.a) == 1 ? 0 : t.a, t.s, t.v}] = t.pt;
        const size_t n = c->n;
        for (size_t ci = 0; ci < nch; ci++) {
            std::vector<rgrp_m> hg;
            std::vector<rterm_m *> owned;
            double b = 0, mm = 0;
            for (size_t g0 = 0; g0 < st.size(); g0 += HE_RNI) {
                const int ni = (int)std::min<size_t>(HE_RNI, st.size() - g0);
                const auto &keys = st[g0]->chunks[ci].ukeys;
                for (int i = 1; i < ni; i++)
                    if (st[g0 + i]->chunks[ci].ukeys.size() != keys.size()) {
                        he_set_error("image-batched split: chunk terms differ");
                        return HE_ESTATE;
                    }
                for (int v0 = 0; v0 < nout; v0 += HE_RVM) {
                    std::vector<rterm_m> ht;
                    for (size_t r = 0; r < keys.size(); r++) {
                        rterm_m T{};
                        bool used = false;
                        for (int v = 0; v < HE_RVM && v0 + v < nout; v++) {
                            auto it = ptm.find({keys[r].first.first, keys[r].first.second, v0 + v});
                            if (it != ptm.end()) { T.pt[v] = it->second; used = true; }
                        }
                        if (!used) continue;
                        for (int i = 0; i < ni; i++) {
                            const auto &kk = st[g0 + i]->chunks[ci].ukeys[r];
                            if (kk.first != keys[r].first) { he_set_error("image-batched split: term order differs"); return HE_ESTATE; }
                            T.U[i] = kk.second;
                        }
                        ht.push_back(T);
                    }
                    rterm_m *d = nullptr;
                    HE_TRY(dev_alloc(&d, std::max<size_t>(1, ht.size())));
                    if (!ht.empty()) HE_CHECK_CUDA(cudaMemcpy(d, ht.data(), ht.size() * sizeof(rterm_m), cudaMemcpyHostToDevice));
                    owned.push_back(d);
                    rgrp_m G{};
                    G.terms = d;
                    G.n_terms = (int)ht.size();
                    G.ni = ni;
                    G.pt_level = a->pt_level;
                    G.nv = std::min(HE_RVM, nout - v0);
                    G.accumulate = ci > 0 ? 1 : 0;
                    int maxext = 0;
                    for (int i = 0; i < ni; i++) {
                        const FusedStage *f = st[g0 + i];
                        G.level[i] = f->level;
                        G.acc[i] = f->facc + (size_t)v0 * 2 * f->ext() * n;
                        maxext = std::max(maxext, f->ext());
                    }
                    hg.push_back(G);
                    for (auto &T : ht) {
                        for (int v = 0; v < HE_RVM; v++)
                            if (T.pt[v]) {
                                if (T.pt[v] != HE_PT_ONE) b += (double)maxext * n * 8;
                                for (int i = 0; i < ni; i++) mm += (double)2 * st[g0 + i]->ext() * n;
                            }
                        for (int i = 0; i < ni; i++) b += (double)2 * st[g0 + i]->ext() * n * 8;
                    }
                    for (int i = 0; i < ni; i++) b += (double)G.nv * 2 * st[g0 + i]->ext() * n * 8;
                }
            }
            rgrp_m *dg = nullptr;
            HE_TRY(dev_alloc(&dg, std::max<size_t>(1, hg.size())));
            if (!hg.empty()) HE_CHECK_CUDA(cudaMemcpy(dg, hg.data(), hg.size() * sizeof(rgrp_m), cudaMemcpyHostToDevice));
            d_mgrps.push_back(dg);
            d_mterms.push_back(owned);
            n_mgrp.push_back((int)hg.size());
            mbytes.push_back(b);
            mmm.push_back(mm);
        }
        splitm_built = true;
        return HE_OK;
    }
    void free_split_m_tables() {
        for (auto *p : d_mgrps) he_free(p);
        for (auto &v : d_mterms)
            for (auto *p : v) he_free(p);
        d_mgrps.clear(); d_mterms.clear(); n_mgrp.clear(); mbytes.clear(); mmm.clear();
        splitm_built = false;
    }
    bool pk_ok() {
        for (auto *f : st)
            if (!f->pk_eligible()) return false;
        return !st.empty();
    }
    size_t pk_need() const {
        size_t b = 0;
        for (auto *f : st) b += f->pk_built ? 0 : f->pk_bytes();
        return b;
    }
    int build_pk() {
        if (d_pk) return HE_OK;
        std::vector<fgrp> h;
        pk_b = pk_mm = 0;
        for (auto *f : st) {
            HE_TRY(f->build_pk());
            for (auto &g : f->pk_groups) {
                h.push_back(g.desc);
                pk_b += g.bytes;
                pk_mm += g.mulmods;
            }
        }
        HE_TRY(dev_alloc(&d_pk, std::max<size_t>(1, h.size())));
        if (!h.empty()) HE_CHECK_CUDA(cudaMemcpy(d_pk, h.data(), h.size() * sizeof(fgrp), cudaMemcpyHostToDevice));
        G_pk = (int)h.size();
        return HE_OK;
    }
    void free_pk() {
        he_free(d_pk);
        d_pk = nullptr;
        G_pk = 0;
        for (auto *f : st) f->free_pk();
    }
    // after a stage's plaintexts changed: drop the pre-keyed tables and tune again on next run
    void reset_pk() {
        he_free(d_pk);
        d_pk = nullptr;
        G_pk = 0;
        if (use_pk) {
            use_pk = false;
            tuned = false;
        }
    }
    int pk_form = HE_KEY_STREAM_PK;                   // or HE_FORM_PK3 (three blocks per SM)
    int launch_pk(cudaStream_t s, int fm = 0) {
        int mb = 0;
        for (auto *f : st) mb = std::max(mb, f->beta());
        return k_ipmac(c, d_pk, G_pk, 1, mb, pk_b, pk_mm, fm ? fm : pk_form, 0, s);
    }
    void free_split_tables() {
        for (auto *p : d_ugrps) he_free(p);
        for (auto *p : d_rgrps) he_free(p);
        d_ugrps.clear(); d_rgrps.clear(); n_ugrp.clear(); n_rgrp.clear();
        ubytes.clear(); rbytes.clear(); rmm.clear();
        split_built = false;
        free_split_m_tables();
    }
    int vmax() const {
        for (auto *f : st)
            if (f->outs.size() >= 2) return 2;
        return 1;
    }

    int build(int Vsel) {
        if (Vsel == V && d_grps) return HE_OK;
        std::vector<fgrp> h;
        bytes = mulmods = 0;
        max_beta = 0;
        for (auto *f : st) {
            HE_TRY(f->build_groups(Vsel));
            for (auto &g : f->groups) {
                h.push_back(g.desc);
                bytes += g.bytes;
                mulmods += g.mulmods;
            }
            max_beta = std::max(max_beta, f->beta());
        }
        he_free(d_grps);
        d_grps = nullptr;
        HE_TRY(dev_alloc(&d_grps, std::max<size_t>(1, h.size())));
        if (!h.empty()) HE_CHECK_CUDA(cudaMemcpy(d_grps, h.data(), h.size() * sizeof(fgrp), cudaMemcpyHostToDevice));
        G = (int)h.size();
        V = Vsel;
        return HE_OK;
    }

    size_t split_need() const {
        size_t b = 0;
        for (auto *f : st) b += f->split_bytes();
        return b;
    }

    int build_split() {
        if (split_built) return HE_OK;
        size_t nch = 0, plan_slot = 0;
        for (auto *f : st) plan_slot = std::max(plan_slot, (size_t)2 * f->ext() * c->n * 8);
        for (auto *f : st) {
            HE_TRY(f->build_split((size_t)2 << 30, plan_slot));
            nch = std::max(nch, f->chunks.size());
        }
        for (size_t ci = 0; ci < nch; ci++) {
            std::vector<ugrp> hu;
            std::vector<rgrp> hr;
            double ub = 0, rb = 0, mm = 0;
            for (auto *f : st) {
                if (ci >= f->chunks.size()) continue;
                auto &ch = f->chunks[ci];
                hu.push_back(ch.udesc);
                for (auto &r : ch.rdesc) hr.push_back(r);
                ub += ch.ubytes;
                rb += ch.rbytes;
                mm += ch.rmm;
            }
            ugrp *du = nullptr;
            rgrp *dr = nullptr;
            HE_TRY(dev_alloc(&du, std::max<size_t>(1, hu.size())));
            HE_TRY(dev_alloc(&dr, std::max<size_t>(1, hr.size())));
            if (!hu.empty()) HE_CHECK_CUDA(cudaMemcpy(du, hu.data(), hu.size() * sizeof(ugrp), cudaMemcpyHostToDevice));
            if (!hr.empty()) HE_CHECK_CUDA(cudaMemcpy(dr, hr.data(), hr.size() * sizeof(rgrp), cudaMemcpyHostToDevice));
            d_ugrps.push_back(du);
            d_rgrps.push_back(dr);
            n_ugrp.push_back((int)hu.size());
            n_rgrp.push_back((int)hr.size());
            ubytes.push_back(ub);
            rbytes.push_back(rb);
            rmm.push_back(mm);
        }
        split_built = true;
        return HE_OK;
    }

    int launch(int fm, cudaStream_t s) { return k_ipmac(c, d_grps, G, V, max_beta, bytes, mulmods, fm, gb, s); }
    int launch_split(cudaStream_t s, bool multi = false) {
        int mb = 0;
        for (auto *f : st) mb = std::max(mb, f->beta());
        for (size_t ci = 0; ci < d_ugrps.size(); ci++) {
            HE_TRY(k_ip_amounts(c, d_ugrps[ci], n_ugrp[ci], mb, ubytes[ci], s));
            if (multi) HE_TRY(k_rmac_m(c, d_mgrps[ci], n_mgrp[ci], mbytes[ci], mmm[ci], s));
            else HE_TRY(k_rmac(c, d_rgrps[ci], n_rgrp[ci], rbytes[ci], rmm[ci], s));
        }
        return HE_OK;
    }

    // candidates: the fused kernel (V outputs per key pass, key stream) and the split form.  The
    // per-thread cp.async ring at one block per SM (HE_KEY_STREAM_CP, and the image-batched split
    // MAC) is left to explicit selection: it shares its construct with kernels that faulted the
    // GPU, and it was never the fastest candidate
    int tune(cudaStream_t s) {
        std::vector<int> forms = {HE_KEY_STREAM_LDG};
        if (max_beta <= 4 && c->d_err) forms.push_back(HE_KEY_STREAM_TMA);
        forms.push_back(HE_KEY_STREAM_LDG1);
        std::vector<int> Vs = {vmax()};
        if (vmax() == 2) Vs.push_back(1);
        bool try_split = false, try_pk = false;
        if (!he_capturing()) {
            size_t fr = 0, tot = 0;
            if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
                try_split = split_need() + ((size_t)4 << 30) < fr;
                const size_t pn = pk_ok() ? pk_need() : 0;
                try_pk = pk_ok() && pn + ((size_t)4 << 30) < fr && pn <= fr / 4;
            }
            cudaGetLastError();
        }
        if ((forms.size() == 1 && Vs.size() == 1 && !try_split && !try_pk) || he_capturing()) {
            // nothing to choose, or no timing possible inside a graph capture: keep the built
            // groups (a captured graph refers to them, so they are never rebuilt afterwards)
            form = forms[0];
            tuned = true;
            return HE_OK;
        }
        cudaEvent_t e0, e1;
        HE_CHECK_CUDA(cudaEventCreate(&e0));
        HE_CHECK_CUDA(cudaEventCreate(&e1));
        float best = 1e30f;
        int bestV = Vs[0], bestF = forms[0];
        bool bestSplit = false;
        char line[1024];
        int pos = snprintf(line, sizeof(line), "%s (%zu stage(s), level %d, %zu outputs):", name.c_str(), st.size(),
                           st.empty() ? 0 : st[0]->level, st.empty() ? (size_t)0 : st[0]->outs.size());
        int rc = HE_OK;
        // time fn() once warm, best of two
        auto time_it = [&](auto fn, float &t) -> int {
            t = 1e30f;
            HE_TRY(fn());
            for (int rep = 0; rep < 2; rep++) {
                float ms = 0;
                if (cudaEventRecord(e0, s) != cudaSuccess) { cudaGetLastError(); he_set_error("autotuner: event"); return HE_ECUDA; }
                HE_TRY(fn());
                if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    cudaGetLastError();
                    he_set_error("autotuner: event timing failed");
                    return HE_ECUDA;
                }
                t = std::min(t, ms);
            }
            return HE_OK;
        };
        for (int Vc : Vs) {
            if ((rc = build(Vc)) != HE_OK) break;
            for (int fm : forms) {
                float t;
                if ((rc = time_it([&]() { return launch(fm, s); }, t)) != HE_OK) break;
                if (pos < (int)sizeof(line))
                    pos += snprintf(line + pos, sizeof(line) - pos, " V=%d %s %.3f ms;", Vc, form_name(fm), t);
                if (t < best) { best = t; bestV = Vc; bestF = fm; bestSplit = false; }
            }
            if (rc != HE_OK) break;
        }
        // shard schedule: batches of groups small enough for their gathered digits to stay in L2
        int bestGb = 0;
        if (rc == HE_OK) rc = build(bestV);
        if (rc == HE_OK && G > 8) {
            for (int gbc : {16, 4}) {
                if (gbc >= G) continue;
                float t;
                gb = gbc;
                rc = time_it([&]() { return launch(bestF, s); }, t);
                gb = 0;
                if (rc != HE_OK) break;
                if (pos < (int)sizeof(line))
                    pos += snprintf(line + pos, sizeof(line) - pos, " V=%d %s gb=%d %.3f ms;", bestV,
                                    form_name(bestF), gbc, t);
                if (t < best) { best = t; bestGb = gbc; }
            }
        }
        bool bestPk = false;
        if (rc == HE_OK && try_pk) {
            rc = build_pk();
            // (HE_KEY_STREAM_PKT, the TMA ring with per-stage release, and HE_KEY_STREAM_PK3L, the L2
            // bulk prefetch two amounts ahead, measured slower than pk3 on the CIFAR layer:
            // explicit selection only)
            for (int fm : {(int)HE_KEY_STREAM_PK, (int)HE_FORM_PK3, (int)HE_FORM_PKP, (int)HE_KEY_STREAM_PK1}) {
                float t;
                if (rc == HE_OK) rc = time_it([&]() { return launch_pk(s, fm); }, t);
                if (rc != HE_OK) break;
                if (pos < (int)sizeof(line))
                    pos += snprintf(line + pos, sizeof(line) - pos, " %s %.3f ms;", pk_name(fm), t);
                if (t < best) { best = t; bestPk = true; bestSplit = false; pk_form = fm; }
            }
        }
        if (rc == HE_OK && try_split) {
            float t;
            rc = build_split();
            if (rc == HE_OK) rc = time_it([&]() { return launch_split(s); }, t);
            if (rc == HE_OK) {
                if (pos < (int)sizeof(line))
                    pos += snprintf(line + pos, sizeof(line) - pos, " split (%zu chunk(s)) %.3f ms;", d_ugrps.size(), t);
                if (t < best) { best = t; bestSplit = true; bestPk = false; }
            }
            if (!use_split_m) free_split_m_tables();
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        HE_TRY(rc);
        if (!bestPk && d_pk) free_pk();                 // give the pre-keyed tables' memory back
        if (bestPk) {
            use_pk = true;
            if (split_built) {
                free_split_tables();
                for (auto *f : st) f->free_split();
            }
        } else if (bestSplit) {
            use_split = true;
            he_free(d_grps);                         // the fused tables are not needed
            d_grps = nullptr;
        } else {
            HE_TRY(build(bestV));
            form = bestF;
            gb = bestGb;
            if (split_built) {                        // give the split form's memory back
                free_split_tables();
                for (auto *f : st) f->free_split();
            }
        }
        tuned = true;
        if (pos < (int)sizeof(line)) {
            if (bestPk) snprintf(line + pos, sizeof(line) - pos, " -> %s", pk_name(pk_form));
            else if (bestSplit) snprintf(line + pos, sizeof(line) - pos, use_split_m ? " -> split-m" : " -> split");
            else snprintf(line + pos, sizeof(line) - pos, " -> V=%d %s gb=%d", bestV, form_name(bestF),
                          bestGb ? bestGb : G);
        }
        he_tune_note(c, line);
        return HE_OK;
    }

    int run(cudaStream_t s) {
        const int opt = c->key_stream;
        for (auto *f : st) HE_TRY(f->hoist(s));
        if (opt == HE_KEY_STREAM_SPLIT || (opt == HE_KEY_STREAM_SPLITM && !splitm_ok())) {   // explicit split form
            HE_TRY(build_split());
            HE_TRY(launch_split(s));
        } else if (opt == HE_KEY_STREAM_SPLITM) {              // explicit image-batched split form
            HE_TRY(build_split_m());
            HE_TRY(launch_split(s, true));
        } else if (is_pk(opt) && pk_ok()) {                     // explicit pre-keyed form
            HE_TRY(build_pk());
            HE_TRY(launch_pk(s, opt));
        } else if (opt != HE_KEY_STREAM_AUTO) {                 // explicit fused form (PK: not eligible)
            const int fm = is_pk(opt) ? HE_KEY_STREAM_LDG : opt;
            if (!d_grps) HE_TRY(build(V ? V : vmax()));
            HE_TRY(launch(fm, s));
        } else {
            if (!d_grps && !use_split && !use_pk) HE_TRY(build(vmax()));
            if (!tuned) HE_TRY(tune(s));
            if (use_pk) HE_TRY(launch_pk(s));
            else if (use_split) HE_TRY(launch_split(s, use_split_m));
            else HE_TRY(launch(form, s));
        }
        for (auto *f : st) HE_TRY(f->moddown(s));
        return HE_OK;
    }
};

// Amount chunks of the split form: each chunk's inner products fit in cap_bytes of U.
static std::vector<std::vector<std::pair<int, std::vector<int>>>> split_plan(
    const FusedStage &f, size_t slot_bytes, size_t cap_bytes) {
    // keyed amount -> sources, in amount order
    std::map<int, std::set<int>> am;                  // amount 0 (no key) comes first
    for (auto &t : f.terms) am[h_galois(f.c, t.a) == 1 ? 0 : t.a].insert(t.s);
    std::vector<std::vector<std::pair<int, std::vector<int>>>> out(1);
    size_t used = 0;
    for (auto &kv : am) {
        const size_t need = kv.second.size() * slot_bytes;
        if (used + need > cap_bytes && !out.back().empty()) {
            out.emplace_back();
            used = 0;
        }
        out.back().push_back({kv.first, std::vector<int>(kv.second.begin(), kv.second.end())});
        used += need;
    }
    return out;
}

size_t FusedStage::split_bytes() const {
    const size_t slot = (size_t)2 * ext() * c->n * 8;
    size_t best = 0;
    for (auto &ch : split_plan(*this, slot, (size_t)2 << 30)) {
        size_t k = 0;
        for (auto &a : ch) k += a.second.size();
        best = std::max(best, k * slot);
    }
    return best;
}

// plan_slot_bytes: the U slot size the amount chunks are planned with (a batch passes its
// largest, so every image of it gets the same chunk boundaries)
int FusedStage::build_split(size_t cap_bytes, size_t plan_slot_bytes) {
    if (split_ready) return HE_OK;
    HE_TRY(build());
    const int nq_ = nq(), ext_ = ext(), beta_ = beta();
    const size_t n = c->n, slot = (size_t)2 * ext_ * n;
    std::vector<const u64 *> Dp(srcs.size());
    for (size_t i = 0; i < srcs.size(); i++)
        Dp[i] = hslot[i] >= 0 ? D_all + (size_t)hslot[i] * beta_ * ext_ * n : nullptr;
    auto plan = split_plan(*this, plan_slot_bytes ? plan_slot_bytes : slot * 8, cap_bytes);
    size_t max_slots = 0;
    for (auto &ch : plan) {
        size_t k = 0;
        for (auto &a : ch) k += a.second.size();
        max_slots = std::max(max_slots, k);
    }
    HE_TRY(dev_alloc(&U, std::max<size_t>(1, max_slots) * slot));
    const int nout = (int)outs.size();
    for (size_t ci = 0; ci < plan.size(); ci++) {
        Chunk ch;
        std::vector<famt> ha;
        std::vector<uent> he;
        std::map<std::pair<int, int>, u64 *> uslot;   // (a, s) -> U slot
        for (auto &a : plan[ci]) {
            famt A;
            A.g = h_galois(c, a.first);
            A.key = nullptr;
            if (A.g != 1) {
                const DeviceKey *k;
                HE_TRY(get_key(c, (int)A.g, &k));
                A.key = k->d;
                ch.ubytes += (double)2 * beta_ * ext_ * n * 8;
            }
            A.e0 = (int)he.size();
            for (int sidx : a.second) {
                u64 *u = U + he.size() * slot;
                he.push_back(uent{Dp[sidx], u, srcs[sidx].d, srcs[sidx].ps, A.g});
                uslot[{a.first, sidx}] = u;
            }
            A.e1 = (int)he.size();
            ha.push_back(A);
            ch.ubytes += (double)(A.e1 - A.e0) * slot * 8;
        }
        HE_TRY(dev_alloc(&ch.d_amt, std::max<size_t>(1, ha.size())));
        HE_TRY(dev_alloc(&ch.d_ent, std::max<size_t>(1, he.size())));
        if (!ha.empty()) HE_CHECK_CUDA(cudaMemcpy(ch.d_amt, ha.data(), ha.size() * sizeof(famt), cudaMemcpyHostToDevice));
        if (!he.empty()) HE_CHECK_CUDA(cudaMemcpy(ch.d_ent, he.data(), he.size() * sizeof(uent), cudaMemcpyHostToDevice));
        ch.udesc = ugrp{ch.d_amt, ch.d_ent, (int)ha.size(), (int)he.size(), level, beta_};
        for (auto &kv : uslot) ch.ukeys.push_back(kv);
        // raised MAC terms per group of HE_RV outputs: this chunk's (a, s) pairs
        for (int v0 = 0; v0 < nout; v0 += HE_RV) {
            std::map<std::pair<int, int>, rterm> tm;
            for (auto &t : terms) {
                if (t.v < v0 || t.v >= v0 + HE_RV) continue;
                const int a = h_galois(c, t.a) == 1 ? 0 : t.a;
                auto it = uslot.find({a, t.s});
                if (it == uslot.end()) continue;              // another chunk
                rterm &r = tm[{a, t.s}];
                r.U = it->second;
                r.pt[t.v - v0] = t.pt;
            }
            std::vector<rterm> ht;
            for (auto &kv : tm) ht.push_back(kv.second);
            rterm *d = nullptr;
            HE_TRY(dev_alloc(&d, std::max<size_t>(1, ht.size())));
            if (!ht.empty()) HE_CHECK_CUDA(cudaMemcpy(d, ht.data(), ht.size() * sizeof(rterm), cudaMemcpyHostToDevice));
            ch.d_terms.push_back(d);
            ch.rdesc.push_back(rgrp{d, (int)ht.size(), level, pt_level, std::min(HE_RV, nout - v0), ci > 0 ? 1 : 0,
                                    facc + (size_t)v0 * 2 * ext_ * n});
            for (auto &r : ht) {
                ch.rbytes += slot * 8.0;
                for (int v = 0; v < HE_RV; v++)
                    if (r.pt[v]) {
                        if (r.pt[v] != HE_PT_ONE) ch.rbytes += (double)ext_ * n * 8;
                        ch.rmm += (double)2 * ext_ * n;
                    }
            }
            ch.rbytes += (double)std::min(HE_RV, nout - v0) * 2 * ext_ * n * 8;
        }
        chunks.push_back(std::move(ch));
    }
    split_ready = true;
    return HE_OK;
}

int FusedStage::build_pk() {
    if (pk_built) return HE_OK;
    HE_TRY(build());
    HE_TRY(he_capture_guard("pre-keyed tables"));
    const size_t n = c->n, kst = (size_t)(c->L + 1 + c->K) * n;
    const int nq_ = nq(), ext_ = ext(), beta_ = beta();
    std::vector<std::map<int, const Term *>> by_out(outs.size());
    for (auto &t : terms) by_out[t.v][t.a] = &t;
    for (size_t v = 0; v < outs.size(); v++) {
        std::vector<famt> ha;
        std::vector<fent> he;
        double bytes = 0, mm = 0;
        for (auto &am : by_out[v]) {
            const Term &T = *am.second;
            famt A{};
            A.g = h_galois(c, am.first);
            const DeviceKey *key = nullptr;
            if (A.g != 1) HE_TRY(get_key(c, (int)A.g, &key));
            fent E{};
            E.s = T.s;
            E.D = hslot[T.s] >= 0 ? D_all + (size_t)hslot[T.s] * beta_ * ext_ * n : nullptr;
            E.src = srcs[T.s].d;
            E.ps = srcs[T.s].ps;
            E.pt[0] = HE_PT_ONE;
            E.pt[1] = nullptr;
            A.key = key ? key->d : nullptr;
            if (T.pt && T.pt != HE_PT_ONE) {
                const auto ck = pk_key(key ? key->d : nullptr, T.pt);
                he_ctx *r = c->root();
                std::lock_guard<std::mutex> lk(r->pk_mu);
                auto it = r->pk_cache.find(ck);
                if (it == r->pk_cache.end()) {
                    he_ctx::PkEntry e;
                    int rc = dev_alloc(&e.Ppt, (size_t)nq_ * n);
                    if (rc == HE_OK && key) rc = dev_alloc(&e.Kp, 2 * beta_ * kst);
                    if (rc == HE_OK)
                        rc = k_prekey(c, key ? key->d : nullptr, T.pt, level, pt_level, key ? beta_ : 0, e.Kp, e.Ppt, 0);
                    if (rc == HE_OK && cudaStreamSynchronize(0) != cudaSuccess) { cudaGetLastError(); rc = HE_ECUDA; }
                    if (rc != HE_OK) { he_free(e.Kp); he_free(e.Ppt); return rc; }
                    it = r->pk_cache.emplace(ck, e).first;
                }
                it->second.refs++;
                pk_refs.push_back(ck);
                A.key = key ? it->second.Kp : nullptr;
                E.pt[0] = it->second.Ppt;
                bytes += (double)nq_ * n * 8;
            }
            if (A.key) bytes += (double)2 * beta_ * ext_ * n * 8;
            mm += (double)ext_ * n * (A.key ? 2 * beta_ : 0) + (double)nq_ * n * 2;
            A.e0 = (int)he.size();
            he.push_back(E);
            A.e1 = (int)he.size();
            ha.push_back(A);
        }
        bytes += (double)nh * beta_ * ext_ * n * 8 / std::max<size_t>(1, outs.size()) +
                 (double)srcs.size() * 2 * nq_ * n * 8 / std::max<size_t>(1, outs.size()) + (double)2 * ext_ * n * 8;
        PkGroup G;
        HE_TRY(dev_alloc(&G.d_amt, std::max<size_t>(1, ha.size())));
        HE_TRY(dev_alloc(&G.d_ent, std::max<size_t>(1, he.size())));
        if (!ha.empty()) HE_CHECK_CUDA(cudaMemcpy(G.d_amt, ha.data(), ha.size() * sizeof(famt), cudaMemcpyHostToDevice));
        if (!he.empty()) HE_CHECK_CUDA(cudaMemcpy(G.d_ent, he.data(), he.size() * sizeof(fent), cudaMemcpyHostToDevice));
        G.desc = fgrp{G.d_amt, G.d_ent, (int)ha.size(), level, beta_, pt_level, 1, facc + v * 2 * ext_ * n};
        G.bytes = bytes;
        G.mulmods = mm;
        pk_groups.push_back(G);
    }
    HE_CHECK_CUDA(cudaStreamSynchronize(0));
    pk_built = true;
    return HE_OK;
}

// Pre-keyed tables hold key (.) plaintext products, so new plaintext contents make them stale:
// release this stage's tables, key any new ones by a fresh epoch, and let the stage's own
// launch tune again (a launch over several stages is reset by its owner).
static std::atomic<uint64_t> g_pk_epoch{0};
void FusedStage::invalidate_pk() {
    free_pk();
    pk_epoch = ++g_pk_epoch;
    if (own) own->reset_pk();
}

FusedStage::~FusedStage() {
    own.reset();
    free_split();
    free_groups();
    free_pk();
    he_free(D_all); he_free(facc); he_free(fconv); he_free(d_md); he_free(htmp); he_free(d_hsrc);
}

int FusedStage::run(cudaStream_t s) {
    HE_TRY(build());
    if (!own) {
        own.reset(new FusedLaunch());
        own->c = c;
        own->st = {this};
        own->name = name;
    }
    return own->run(s);
}

// ================================================================================ pooling
struct he_pool {
    he_ctx *c = nullptr;
    PoolPlanH P;
    int level = 0, ns = 0;
    size_t pw0 = 0, pw1 = 0, pw2 = 0;
    // buffers: X[ns] (pw0), W[ns] (pw0), Y[ns] (pw0: MAC at level, rescaled in place),
    // Z[ns] (pw1), S[groups] (pw2); rotated copies per stage
    u64 *X = nullptr, *Wb = nullptr, *Yb = nullptr, *Zb = nullptr, *Sb = nullptr;
    u64 *rotS = nullptr, *rotH = nullptr, *rotV = nullptr, *rotC = nullptr, *rotD = nullptr;
    RotSet rs_S, rs_H, rs_V, rs_C, rs_D;
    u64 *hpts = nullptr, *vpts = nullptr;     // masks over Q_l u P (stride pe0 / pe1)
    size_t pe0 = 0, pe1 = 0;
    std::vector<int> h_idx, v_idx;
    int n_hpt = 0, n_vpt = 0;
    mac_term *d_hterms = nullptr, *d_vterms = nullptr;
    FusedStage f_S, f_H, f_V, f_C, f_D;     // HE_FUSED stages (built on first use)
    bool shared_masks = false;               // forks share the parent's mask plaintexts
    bool rot_ready = false;                  // per-rotation buffers of HE_PLAIN / HE_BATCHED
    ~he_pool() {
        he_free(X); he_free(Wb); he_free(Yb); he_free(Zb); he_free(Sb);
        he_free(rotS); he_free(rotH); he_free(rotV); he_free(rotC); he_free(rotD);
        he_free(d_hterms); he_free(d_vterms);
        if (!shared_masks) { he_free(hpts); he_free(vpts); }
    }
};

static int dedupe_upload(he_ctx *c, const std::vector<std::vector<std::vector<double>>> &mk, int ns,
                         int lv, u64 **dst, std::vector<int> &idx, int &count) {
    // stored over Q_lv u P so the fused stages can use them; the plain MAC reads the Q limbs
    std::vector<const double *> uniq;
    std::unordered_map<uint64_t, std::vector<int>> seen;
    idx.assign(mk.size() * ns, -1);
    for (size_t a = 0; a < mk.size(); a++)
        for (int u = 0; u < ns; u++) {
            const std::vector<double> &v = mk[a][u];
            uint64_t h = 1469598103934665603ull;
            for (int i = 0; i < c->N; i++) {
                uint64_t bits;
                memcpy(&bits, &v[i], 8);
                h = (h ^ bits) * 1099511628211ull;
            }
            int found = -1;
            for (int cand : seen[h])
                if (!memcmp(uniq[cand], v.data(), (size_t)c->N * 8)) { found = cand; break; }
            if (found < 0) {
                found = (int)uniq.size();
                uniq.push_back(v.data());
                seen[h].push_back(found);
            }
            idx[a * ns + u] = found;
        }
    count = (int)uniq.size();
    HE_TRY(dev_alloc(dst, (size_t)count * (lv + 1 + c->K) * c->n));
    return upload_plaintexts(c, uniq, uniq.size(), (double)c->primes[lv], lv, *dst, nullptr, true);
}

// stage buffers every mode uses
static int pool_runtime(he_pool *p) {
    const PoolPlanH &P = p->P;
    const int ns = p->ns;
    HE_TRY(dev_alloc(&p->X, (size_t)ns * 2 * p->pw0));
    HE_TRY(dev_alloc(&p->Wb, (size_t)ns * 2 * p->pw0));
    HE_TRY(dev_alloc(&p->Yb, (size_t)ns * 2 * p->pw0));
    HE_TRY(dev_alloc(&p->Zb, (size_t)ns * 2 * p->pw1));
    HE_TRY(dev_alloc(&p->Sb, P.groups.size() * 2 * p->pw2));
    HE_TRY(dev_alloc(&p->rotD, P.dup.size() * 2 * p->pw2));
    return HE_OK;
}

// buffers, rotation sets and MAC tables of the per-rotation modes (HE_PLAIN / HE_BATCHED)
static int pool_rot_runtime(he_pool *p) {
    if (p->rot_ready) return HE_OK;
    he_ctx *c = p->c;
    const PoolPlanH &P = p->P;
    const int ns = p->ns, level = p->level;
    const size_t pw0 = p->pw0, pw1 = p->pw1, pw2 = p->pw2;
    const size_t nS = P.pre.size(), nH = P.h_amt.size(), nV = P.v_amt.size(), nG = P.groups.size();
    HE_TRY(dev_alloc(&p->rotS, (size_t)ns * nS * 2 * pw0));
    HE_TRY(dev_alloc(&p->rotH, (size_t)ns * nH * 2 * pw0));
    HE_TRY(dev_alloc(&p->rotV, (size_t)ns * nV * 2 * pw1));
    HE_TRY(dev_alloc(&p->rotC, (size_t)ns * 2 * pw2));
    for (RotSet *rs : {&p->rs_S, &p->rs_H, &p->rs_V, &p->rs_C, &p->rs_D}) rs->c = c;
    p->rs_S.level = level;
    p->rs_H.level = level;
    p->rs_V.level = level - 1;
    p->rs_C.level = level - 2;
    p->rs_D.level = level - 2;
    u64 *hsrc = nS ? p->Wb : p->X;
    for (int u = 0; u < ns; u++) {
        p->rs_S.src.push_back({p->X + (size_t)u * 2 * pw0, pw0});
        p->rs_H.src.push_back({hsrc + (size_t)u * 2 * pw0, pw0});
        p->rs_V.src.push_back({p->Yb + (size_t)u * 2 * pw0, pw0});
        p->rs_C.src.push_back({p->Zb + (size_t)u * 2 * pw1, pw1});
        for (size_t a = 0; a < nS; a++) p->rs_S.add(u, P.pre[a], p->rotS + ((size_t)u * nS + a) * 2 * pw0, pw0);
        for (size_t a = 0; a < nH; a++) p->rs_H.add(u, P.h_amt[a], p->rotH + ((size_t)u * nH + a) * 2 * pw0, pw0);
        for (size_t a = 0; a < nV; a++) p->rs_V.add(u, P.v_amt[a], p->rotV + ((size_t)u * nV + a) * 2 * pw1, pw1);
    }
    for (size_t g = 0; g < nG; g++)
        for (auto &e : P.groups[g]) p->rs_C.add(e.first, e.second, p->rotC + (size_t)e.first * 2 * pw2, pw2);
    if (P.dup.size() > 1) {
        p->rs_D.src.push_back({p->Sb, pw2});
        for (size_t k = 0; k < P.dup.size(); k++) p->rs_D.add(0, P.dup[k], p->rotD + k * 2 * pw2, pw2);
    }
    std::vector<mac_term> th, tv;
    for (int u = 0; u < ns; u++) {
        for (size_t a = 0; a < nH; a++)
            th.push_back({p->hpts + (size_t)p->h_idx[a * ns + u] * p->pe0, p->rotH + ((size_t)u * nH + a) * 2 * pw0, pw0});
        for (size_t a = 0; a < nV; a++)
            tv.push_back({p->vpts + (size_t)p->v_idx[a * ns + u] * p->pe1, p->rotV + ((size_t)u * nV + a) * 2 * pw1, pw1});
    }
    HE_TRY(dev_alloc(&p->d_hterms, th.size()));
    HE_TRY(dev_alloc(&p->d_vterms, tv.size()));
    HE_CHECK_CUDA(cudaMemcpy(p->d_hterms, th.data(), th.size() * sizeof(mac_term), cudaMemcpyHostToDevice));
    HE_CHECK_CUDA(cudaMemcpy(p->d_vterms, tv.data(), tv.size() * sizeof(mac_term), cudaMemcpyHostToDevice));
    p->rot_ready = true;
    return HE_OK;
}

static void pool_sizes(he_pool *p, he_ctx *c, int level) {
    p->c = c;
    p->level = level;
    p->pw0 = (size_t)(level + 1) * c->n;
    p->pw1 = (size_t)level * c->n;
    p->pw2 = (size_t)(level - 1) * c->n;
    p->pe0 = (size_t)(level + 1 + c->K) * c->n;
    p->pe1 = (size_t)(level + c->K) * c->n;
}

static int pool_build(he_ctx *c, const Lay &lin, int level, bool select, he_pool **out) {
    if (level < 2) { he_set_error("pooling needs two levels"); return HE_ELEVEL; }
    if (check_layout(lin, c->N) != HE_OK) return HE_EINVAL;
    std::unique_ptr<he_pool> p(new he_pool());
    pool_sizes(p.get(), c, level);
    HE_TRY(plan_pool(lin, select, p->P));
    p->ns = lin.ns;
    HE_TRY(dedupe_upload(c, p->P.h_mask, p->ns, level, &p->hpts, p->h_idx, p->n_hpt));
    HE_TRY(dedupe_upload(c, p->P.v_mask, p->ns, level - 1, &p->vpts, p->v_idx, p->n_vpt));
    p->P.h_mask.clear();
    p->P.v_mask.clear();
    HE_TRY(pool_runtime(p.get()));
    *out = p.release();
    return HE_OK;
}

static int pool_fork(const he_pool *src, he_ctx *c, he_pool **out) {
    if (c->root() != src->c->root()) { he_set_error("fork: contexts do not share a root"); return HE_ESTATE; }
    std::unique_ptr<he_pool> p(new he_pool());
    pool_sizes(p.get(), c, src->level);
    p->P = src->P;
    p->ns = src->ns;
    p->hpts = src->hpts;
    p->vpts = src->vpts;
    p->h_idx = src->h_idx;
    p->v_idx = src->v_idx;
    p->n_hpt = src->n_hpt;
    p->n_vpt = src->n_vpt;
    p->shared_masks = true;
    HE_TRY(pool_runtime(p.get()));
    *out = p.release();
    return HE_OK;
}

static int pool_run_fused(he_ctx *c, he_pool *p, he_ct *const *in, he_ct **out, cudaStream_t s);

static int pool_run(he_ctx *c, he_pool *p, he_ct *const *in, he_ct **out, int mode, cudaStream_t s) {
    if (mode == HE_FUSED) return pool_run_fused(c, p, in, out, s);
    const int ns = p->ns, lv = p->level;
    const size_t pw0 = p->pw0, pw1 = p->pw1, pw2 = p->pw2;
    const PoolPlanH &P = p->P;
    const double scale = in[0]->scale;
    for (int u = 0; u < ns; u++) {
        if (!in[u] || in[u]->ctx != c || in[u]->level != lv || in[u]->scale != scale) {
            he_set_error("pool input %d: level or scale mismatch", u);
            return HE_ELEVEL;
        }
        HE_TRY(k_copy_limbs(p->X + (size_t)u * 2 * pw0, pw0, in[u]->d, in[u]->pstride, pw0, 2, s));
    }
    const size_t nS = P.pre.size(), nH = P.h_amt.size(), nV = P.v_amt.size();
    if (nS) {                                                          // S
        HE_TRY(p->rs_S.run(mode, s));
        for (int u = 0; u < ns; u++) {
            u64 *acc = p->Wb + (size_t)u * 2 * pw0;
            HE_TRY(k_copy_limbs(acc, pw0, p->rotS + (size_t)u * nS * 2 * pw0, pw0, pw0, 2, s));
            for (size_t a = 1; a < nS; a++)
                HE_TRY(k_add_raw(c, acc, pw0, p->rotS + ((size_t)u * nS + a) * 2 * pw0, pw0, lv + 1, 2, false, s));
        }
    }
    HE_TRY(p->rs_H.run(mode, s));                                      // H
    double sH = scale;
    for (int u = 0; u < ns; u++) {
        u64 *y = p->Yb + (size_t)u * 2 * pw0;
        HE_TRY(k_mac(c, p->d_hterms + (size_t)u * nH, (int)nH, y, pw0, lv, false, s));
        he_ct t = view(c, y, pw0, lv, scale * (double)c->primes[lv]);
        HE_TRY(he_rescale(c, &t, s));
        sH = t.scale;
    }
    HE_TRY(p->rs_V.run(mode, s));                                      // V
    double sV = sH;
    for (int u = 0; u < ns; u++) {
        u64 *z = p->Zb + (size_t)u * 2 * pw1;
        HE_TRY(k_mac(c, p->d_vterms + (size_t)u * nV, (int)nV, z, pw1, lv - 1, false, s));
        he_ct t = view(c, z, pw1, lv - 1, sH * (double)c->primes[lv - 1]);
        HE_TRY(he_rescale(c, &t, s));
        sV = t.scale;
    }
    HE_TRY(p->rs_C.run(mode, s));                                      // C
    for (size_t g = 0; g < P.groups.size(); g++) {
        u64 *acc = p->Sb + g * 2 * pw2;
        const auto &grp = P.groups[g];
        HE_TRY(k_copy_limbs(acc, pw2, p->rotC + (size_t)grp[0].first * 2 * pw2, pw2, pw2, 2, s));
        for (size_t q = 1; q < grp.size(); q++)
            HE_TRY(k_add_raw(c, acc, pw2, p->rotC + (size_t)grp[q].first * 2 * pw2, pw2, lv - 1, 2, false, s));
    }
    const int lo = lv - 2;
    if (P.dup.size() > 1) {                                            // duplicate
        HE_TRY(p->rs_D.run(mode, s));
        HE_TRY(ensure_ct(c, out[0], lo));
        HE_TRY(k_copy_limbs(out[0]->d, out[0]->pstride, p->rotD, pw2, pw2, 2, s));
        for (size_t k = 1; k < P.dup.size(); k++)
            HE_TRY(k_add_raw(c, out[0]->d, out[0]->pstride, p->rotD + k * 2 * pw2, pw2, lo + 1, 2, false, s));
        out[0]->scale = sV;
    } else {
        for (size_t g = 0; g < P.groups.size(); g++) {
            HE_TRY(ensure_ct(c, out[g], lo));
            HE_TRY(k_copy_limbs(out[g]->d, out[g]->pstride, p->Sb + g * 2 * pw2, pw2, pw2, 2, s));
            out[g]->scale = sV;
        }
    }
    return HE_OK;
}

static int pool_prepare_fused(he_pool *p) {
    if (p->f_H.c) return HE_OK;
    he_ctx *c = p->c;
    const int ns = p->ns, lv = p->level;
    const PoolPlanH &P = p->P;
    const size_t pw0 = p->pw0, pw1 = p->pw1, pw2 = p->pw2;
    const size_t nH = P.h_amt.size(), nV = P.v_amt.size();
    for (FusedStage *f : {&p->f_S, &p->f_H, &p->f_V, &p->f_C, &p->f_D}) f->c = c;
    char nm[64];
    const char *tag[5] = {"S (ones conv)", "H (horizontal)", "V (vertical)", "C (consolidate)", "D (duplicate)"};
    FusedStage *fs[5] = {&p->f_S, &p->f_H, &p->f_V, &p->f_C, &p->f_D};
    for (int k = 0; k < 5; k++) {
        snprintf(nm, sizeof(nm), "pool %dx%d %s", p->P.lin.m, p->P.lin.m, tag[k]);
        fs[k]->name = nm;
    }
    p->f_S.level = p->f_H.level = lv;
    p->f_V.level = lv - 1;
    p->f_C.level = p->f_D.level = lv - 2;
    u64 *hsrc = P.pre.empty() ? p->X : p->Wb;
    for (int u = 0; u < ns; u++) {
        p->f_S.add_src(p->X + (size_t)u * 2 * pw0, pw0);
        p->f_S.add_out(p->Wb + (size_t)u * 2 * pw0, pw0);
        for (int a : P.pre) p->f_S.add_term(u, u, a, HE_PT_ONE);
        p->f_H.add_src(hsrc + (size_t)u * 2 * pw0, pw0);
        p->f_H.add_out(p->Yb + (size_t)u * 2 * pw0, pw0);
        for (size_t a = 0; a < nH; a++)
            p->f_H.add_term(u, u, P.h_amt[a], p->hpts + (size_t)p->h_idx[a * ns + u] * p->pe0);
        p->f_V.add_src(p->Yb + (size_t)u * 2 * pw0, pw0);
        p->f_V.add_out(p->Zb + (size_t)u * 2 * pw1, pw1);
        for (size_t a = 0; a < nV; a++)
            p->f_V.add_term(u, u, P.v_amt[a], p->vpts + (size_t)p->v_idx[a * ns + u] * p->pe1);
        p->f_C.add_src(p->Zb + (size_t)u * 2 * pw1, pw1);
    }
    for (size_t g = 0; g < P.groups.size(); g++) {
        p->f_C.add_out(p->Sb + g * 2 * pw2, pw2);
        for (auto &e : P.groups[g]) p->f_C.add_term((int)g, e.first, e.second, HE_PT_ONE);
    }
    if (P.dup.size() > 1) {
        p->f_D.add_src(p->Sb, pw2);
        p->f_D.add_out(p->rotD, pw2);
        for (int a : P.dup) p->f_D.add_term(0, 0, a, HE_PT_ONE);
        HE_TRY(p->f_D.build());
    }
    if (!P.pre.empty()) HE_TRY(p->f_S.build());
    HE_TRY(p->f_H.build());
    HE_TRY(p->f_V.build());
    return p->f_C.build();
}

static int pool_run_fused(he_ctx *c, he_pool *p, he_ct *const *in, he_ct **out, cudaStream_t s) {
    const int ns = p->ns, lv = p->level;
    const size_t pw0 = p->pw0, pw1 = p->pw1, pw2 = p->pw2;
    const PoolPlanH &P = p->P;
    const double scale = in[0]->scale;
    for (int u = 0; u < ns; u++) {
        if (!in[u] || in[u]->ctx != c || in[u]->level != lv || in[u]->scale != scale) {
            he_set_error("pool input %d: level or scale mismatch", u);
            return HE_ELEVEL;
        }
        HE_TRY(k_copy_limbs(p->X + (size_t)u * 2 * pw0, pw0, in[u]->d, in[u]->pstride, pw0, 2, s));
    }
    if (!P.pre.empty()) HE_TRY(p->f_S.run(s));
    HE_TRY(p->f_H.run(s));
    double sH = scale;
    for (int u = 0; u < ns; u++) {
        he_ct t = view(c, p->Yb + (size_t)u * 2 * pw0, pw0, lv, scale * (double)c->primes[lv]);
        HE_TRY(he_rescale(c, &t, s));
        sH = t.scale;
    }
    HE_TRY(p->f_V.run(s));
    double sV = sH;
    for (int u = 0; u < ns; u++) {
        he_ct t = view(c, p->Zb + (size_t)u * 2 * pw1, pw1, lv - 1, sH * (double)c->primes[lv - 1]);
        HE_TRY(he_rescale(c, &t, s));
        sV = t.scale;
    }
    HE_TRY(p->f_C.run(s));
    const int lo = lv - 2;
    if (P.dup.size() > 1) {
        HE_TRY(p->f_D.run(s));
        HE_TRY(ensure_ct(c, out[0], lo));
        HE_TRY(k_copy_limbs(out[0]->d, out[0]->pstride, p->rotD, pw2, pw2, 2, s));
        out[0]->scale = sV;
    } else {
        for (size_t g = 0; g < P.groups.size(); g++) {
            HE_TRY(ensure_ct(c, out[g], lo));
            HE_TRY(k_copy_limbs(out[g]->d, out[g]->pstride, p->Sb + g * 2 * pw2, pw2, pw2, 2, s));
            out[g]->scale = sV;
        }
    }
    return HE_OK;
}

static int pool_prepare(he_pool *p, int mode) {
    if (mode == HE_FUSED) return pool_prepare_fused(p);
    HE_TRY(pool_rot_runtime(p));
    for (RotSet *rs : {&p->rs_S, &p->rs_H, &p->rs_V, &p->rs_C, &p->rs_D}) {
        if (mode == HE_BATCHED) HE_TRY(rs->prepare_batched());
        else HE_TRY(rs->resolve_keys());
    }
    return HE_OK;
}

static void collect_rotations(const he_pool *p, std::vector<int> &v) {
    const PoolPlanH &P = p->P;
    for (int a : P.pre) v.push_back(a);
    for (int a : P.h_amt) v.push_back(a);
    for (int a : P.v_amt) v.push_back(a);
    for (auto &g : P.groups)
        for (auto &e : g) v.push_back(e.second);
    for (int a : P.dup) v.push_back(a);
}

extern "C" int he_pool_create(he_ctx *c, const he_layout *in, int level, he_pool **out) {
    if (!c || !in || !out) { he_set_error("null argument"); return HE_EINVAL; }
    if (level < 2 || level > c->L) { he_set_error("he_pool_create: level %d out of range", level); return HE_ELEVEL; }
    return pool_build(c, from_c(*in), level, false, out);
}
extern "C" void he_pool_destroy(he_pool *p) {
    if (p) { cudaDeviceSynchronize(); delete p; }
}
extern "C" int he_pool_out_layout(const he_pool *p, he_layout *out) {
    if (!p || !out) return HE_EINVAL;
    return to_c(p->P.lout, out);
}
static int distinct_nonzero(he_ctx *c, std::vector<int> v, int32_t *amounts, size_t cap) {
    std::vector<int> r;
    std::vector<u64> gs;
    for (int a : v) {
        u64 g = h_galois(c, a);
        if (g == 1 || std::find(gs.begin(), gs.end(), g) != gs.end()) continue;
        gs.push_back(g);
        r.push_back(a);
    }
    for (size_t i = 0; i < r.size() && i < cap; i++) amounts[i] = r[i];
    return (int)r.size();
}
extern "C" int he_pool_rotations(const he_pool *p, int32_t *amounts, size_t cap) {
    if (!p) return HE_EINVAL;
    std::vector<int> v;
    collect_rotations(p, v);
    return distinct_nonzero(p->c, v, amounts, cap);
}
extern "C" int he_pool_n_masks(const he_pool *p, int *n_h, int *n_v) {
    if (!p) return HE_EINVAL;
    if (n_h) *n_h = (int)p->P.h_amt.size();
    if (n_v) *n_v = (int)p->P.v_amt.size();
    return HE_OK;
}

static int import_masks(he_pool *p, const int64_t *m, size_t n_amt, const std::vector<int> &idx, int count,
                        int lv, u64 *dst) {
    he_ctx *c = p->c;
    std::vector<int64_t> pick((size_t)count * c->n);
    std::vector<char> done(count, 0);
    for (size_t a = 0; a < n_amt; a++)
        for (int u = 0; u < p->ns; u++) {
            int k = idx[a * p->ns + u];
            if (done[k]) continue;
            memcpy(pick.data() + (size_t)k * c->n, m + (a * p->ns + u) * (size_t)c->n, (size_t)c->n * 8);
            done[k] = 1;
        }
    std::vector<const double *> none;
    return upload_plaintexts(c, none, (size_t)count, 0.0, lv, dst, pick.data(), true);
}

extern "C" int he_pool_import_plaintexts(he_pool *p, const int64_t *h, const int64_t *v) {
    if (!p) return HE_EINVAL;
    if (h) HE_TRY(import_masks(p, h, p->P.h_amt.size(), p->h_idx, p->n_hpt, p->level, p->hpts));
    if (v) HE_TRY(import_masks(p, v, p->P.v_amt.size(), p->v_idx, p->n_vpt, p->level - 1, p->vpts));
    for (FusedStage *f : {&p->f_S, &p->f_H, &p->f_V, &p->f_C, &p->f_D}) f->invalidate_pk();
    return HE_OK;
}

extern "C" int he_pool_run(he_ctx *c, he_pool *p, he_ct *const *in, he_ct **out, int mode, void *stream) {
    if (!c || !p || !in || !out || p->c != c || mode < HE_PLAIN || mode > HE_FUSED) {
        he_set_error("he_pool_run: bad argument");
        return HE_EINVAL;
    }
    HE_TRY(pool_prepare(p, mode));
    return pool_run(c, p, in, out, mode, (cudaStream_t)stream);
}

// ================================================================================ convolution
struct ConvBatch;
struct FactoredConv;
struct he_conv {
    he_ctx *c = nullptr;
    Lay lin, lout;
    std::vector<double> W, bias;
    int co = 0, ci = 0, kh = 0, kw = 0, pad = 0, stride = 1, level = 0;
    double in_scale = 1.0, mid_scale = 1.0;
    size_t pw = 0;
    std::vector<int> tu, tv, ta;                 // terms in plan order
    std::vector<int> term_off;                   // [n_out + 1]
    std::map<long long, int> slot;               // u*N + a -> rotation slot (amount != 0)
    size_t pe = 0;                               // plaintext stride: Q_l u P limbs
    u64 *R = nullptr;                            // [n_in][2][pw] input copies
    u64 *Rrot = nullptr;                         // [slots][2][pw] rotations (per-rotation modes)
    u64 *pts = nullptr, *bias_pts = nullptr, *acc = nullptr;
    mac_term *d_terms = nullptr;
    RotSet rot;
    bool rot_ready = false, shared_pts = false;
    he_pool *pool = nullptr;
    std::vector<he_ct *> mid;
    FusedStage fused;                            // HE_FUSED: built on first use
    std::unique_ptr<ConvBatch> batch;            // he_conv_run_batch: buffers of the last signature
    std::unique_ptr<FactoredConv> fc;            // set: the factored channel-shard form
    std::map<std::pair<int, uint64_t>, u64 *> bias_by;   // (level, output scale) -> bias addends
    // baby-step giant-step form: term t reads rot_{tt[t]}(X_u) into the partial sum ts[t];
    // partial sum i is S_{sv[i], sg[i]}, rotated by sg[i] into output shard sv[i]
    bool bsgs = false;
    int bsgs_k = 0;                              // giant stride in blocks
    std::vector<int> tt, ts, sv, sg, s_off;      // s_off: [nS + 1] term range of each partial sum
    u64 *Sb = nullptr, *Gb = nullptr;            // [nS][2][pw] partial sums, rotated partial sums
    RotSet grot;                                 // per-rotation modes: giant rotations
    bool grot_ready = false;
    FusedStage fusedG;                           // HE_FUSED: giant stage
    int term_amt(size_t t) const { return bsgs ? tt[t] : ta[t]; }   // rotation a term's input takes
    u64 *rot_ptr(int u, int a) {
        return a == 0 ? R + (size_t)u * 2 * pw : Rrot + (size_t)slot[(long long)u * c->N + a] * 2 * pw;
    }
    ~he_conv();
};

// Baby-step giant-step split of a diagonal amount: a = r B + s with s the residue of a modulo
// the block length B taken in [-B/2, B/2) (the tap's row and column shift) and r the channel
// offset in blocks (r m^2 of Eqs. 2-5); with a giant stride of k blocks the baby amount is
// t = (r mod k) B + s and the giant amount g = (r - r mod k) B (mod N).
static void bsgs_split(int a, int B, int N, int k, int &g, int &t) {
    int s = a % B;
    if (2 * s >= B) s -= B;
    const int nb = N / B;
    const int r = (((a - s) / B) % nb + nb) % nb;
    g = (int)((long long)(r - r % k) * B % N);
    t = (((r % k) * B + s) % N + N) % N;
}

// Modelled time (us) of the BSGS form with giant stride k at a level: the key and raised-digit
// streams at an effective 4.5 TB/s, and each ModUp (nq INTT + beta ext NTT limbs) and ModDown
// (2 (K + nq) limbs) at 1.3 us per 2^16-word limb transform with its base conversion (both
// rates as measured on the CIFAR-layer and ResNet-block convolutions).  terms: (v, u, a).
static double bsgs_cost(const he_ctx *c, const Lay &lin, int level, const std::vector<std::array<int, 3>> &terms,
                        int n_out, int k) {
    std::set<int> amt_b, amt_g, src_b;
    std::set<std::pair<int, int>> ent_b, S, grot;
    for (auto &x : terms) {
        int g, t;
        bsgs_split(x[2], lin.B, lin.N, k, g, t);
        S.insert({x[0], g});
        if (t != 0) { amt_b.insert(t); ent_b.insert({x[1], t}); src_b.insert(x[1]); }
        if (g != 0) { amt_g.insert(g); grot.insert({x[0], g}); }
    }
    const double nq = level + 1, ext = nq + c->K, beta = (level + c->alpha) / c->alpha;
    const double limb = (double)c->n * 8, tlimb = 1.3e-6 * c->n / 65536.0;
    const double keys = (double)(amt_b.size() + amt_g.size()) * 2 * beta * ext;
    const double ents = (double)(ent_b.size() + grot.size()) * 3 * ext + (double)(ent_b.size() + grot.size()) * beta * ext;
    const double hbm = (keys + ents) * limb / 4.5e12;
    const double alu = ((double)(src_b.size() + grot.size()) * (nq + beta * ext) +
                        (double)(S.size() + n_out) * 2 * (c->K + nq)) * tlimb;
    return (hbm + alu) * 1e6;
}

static int conv_bias_int(he_conv *cv, int v, double scale, std::vector<int64_t> &m) {
    std::vector<double> z(cv->c->N, 0.0);
    for (int i = 0; i < cv->c->N; i++) {
        SlotInfo s = slot_info(cv->lout, v, i);
        if (s.valid && !cv->bias.empty()) z[i] = cv->bias[s.ch];
    }
    m.resize(cv->c->n);
    encode_slots(z.data(), cv->c->n, scale, m.data());
    return HE_OK;
}

// ================================================================================ factored conv
// Channel-shard convolution in two stages (Eq. 7 with the weights taken out of the masks):
// stage 1  Y_{f,h,t} = sum_{h'} B_{h,h',t} (.) rot_{a_t}(X_{f,h'})   binary masks at scale q_l,
//          rescale;
// stage 2  out_{o,h} = sum_{f,t} round(W[o][f][t] q_{l-1}) Y_{f,h,t}   integer scalars, rescale,
//          bias.
// Every shard holds R = N/M rows of one channel (H = M/R shards per channel); own and
// neighbour reads of a tap share the amount a_t = ((k - pad) M + (l - pad)) mod N, and the masks
// depend on (h, h', t) only, so there are at most 2 H T of them instead of co ci H T diagonals.
struct FactoredConv {
    int H = 0, T = 0, nY = 0, n_masks = 0;
    std::vector<int> amt;                        // per tap
    std::vector<std::array<int, 3>> mkey;        // (h, h_src, t), sorted
    u64 *masks = nullptr;                        // [n_masks][l+1+K][n] Montgomery NTT, scale q_l
    u64 *Wm = nullptr;                           // [l][co][ci T] Montgomery residues (limbs 0..l-1)
    u64 *Y = nullptr;                            // [nY][2][pw] stage-1 outputs
    u64 *rt = nullptr;                           // rescale scratch [2 max(nY, n_out)][l][n]
    std::vector<int> yoff, ts, ta, tm;           // stage-1 terms per Y: source, amount, mask
    FusedStage fy;                               // HE_FUSED stage 1
    RotSet ry;                                   // per-rotation stage 1
    u64 *Rrot = nullptr;
    std::map<int, int> rslot;                    // (u * N + a) -> rotation slot
    mac_term *d_terms = nullptr;
    bool rot_ready = false;
    ~FactoredConv() { he_free(masks); he_free(Wm); he_free(Y); he_free(rt); he_free(Rrot); he_free(d_terms); }
};

// the masks B_{h,h',t} (sorted by key) and the tap amounts
static int factored_masks(const he_conv *cv, std::vector<std::array<int, 3>> &keys,
                          std::vector<std::vector<double>> &mvals, std::vector<int> &amt) {
    const Lay &L = cv->lin;
    const int M = L.M, N = L.N, R = L.rows(), H = M / R;
    std::map<std::array<int, 3>, std::vector<double>> mk;
    amt.clear();
    for (int k = 0; k < cv->kh; k++)
        for (int l = 0; l < cv->kw; l++) {
            const int t = k * cv->kw + l;
            const int a = (int)((((long long)(k - cv->pad) * M + (l - cv->pad)) % N + N) % N);
            amt.push_back(a);
            for (int h = 0; h < H; h++)
                for (int i = 0; i < N; i++) {
                    SlotInfo si = slot_info(cv->lout, h, i);      // shard h of output channel 0
                    const int ys = si.y + k - cv->pad, xs = si.x + l - cv->pad;
                    if (!si.valid || ys < 0 || ys >= L.m || xs < 0 || xs >= L.m) continue;
                    const int hs = ys / R;
                    const int j = (ys - hs * R) * M + xs;
                    if (((j - i) % N + N) % N != a) { he_set_error("factored conv: amounts disagree"); return HE_ESTATE; }
                    auto &v = mk[{h, hs, t}];
                    if (v.empty()) v.assign(N, 0.0);
                    v[i] = 1.0;
                }
        }
    keys.clear();
    mvals.clear();
    for (auto &kv : mk) {
        keys.push_back(kv.first);
        mvals.push_back(std::move(kv.second));
    }
    return HE_OK;
}

static int factored_plan(he_conv *cv, std::vector<std::vector<double>> &mvals) {
    he_ctx *c = cv->c;
    FactoredConv &F = *cv->fc;
    const Lay &L = cv->lin;
    F.H = L.M / L.rows();
    F.T = cv->kh * cv->kw;
    F.nY = cv->ci * F.H * F.T;
    HE_TRY(factored_masks(cv, F.mkey, mvals, F.amt));
    F.n_masks = (int)F.mkey.size();
    // stage-1 terms per Y = (f, h, t)
    for (int f = 0; f < cv->ci; f++)
        for (int h = 0; h < F.H; h++)
            for (int t = 0; t < F.T; t++) {
                F.yoff.push_back((int)F.ts.size());
                for (int m = 0; m < F.n_masks; m++)
                    if (F.mkey[m][0] == h && F.mkey[m][2] == t) {
                        F.ts.push_back(f * F.H + F.mkey[m][1]);
                        F.ta.push_back(F.amt[t]);
                        F.tm.push_back(m);
                    }
            }
    F.yoff.push_back((int)F.ts.size());
    // stage-2 scalars round(w q_{l-1}), residues mod q_0..q_{l-1} in Montgomery form
    const int l1 = cv->level - 1, nin = cv->ci * F.T;
    std::vector<u64> wm((size_t)(l1 + 1) * cv->co * nin);
    const double ql1 = (double)c->primes[l1];
    for (int o = 0; o < cv->co; o++)
        for (int f = 0; f < cv->ci; f++)
            for (int t = 0; t < F.T; t++) {
                const double w = cv->W[(((size_t)o * cv->ci + f) * cv->kh + t / cv->kw) * cv->kw + t % cv->kw];
                const double r = std::round(w * ql1);               // half away from zero
                if (!(std::fabs(r) < 9.0e18)) { he_set_error("factored conv: weight too large"); return HE_EINVAL; }
                const long long wi = (long long)r;
                for (int i = 0; i <= l1; i++) {
                    const u64 q = c->primes[i];
                    const u64 res = wi >= 0 ? (u64)wi % q : (q - (u64)(-wi) % q) % q;
                    wm[((size_t)i * cv->co + o) * nin + f * F.T + t] = (u64)(((u128)res << 64) % q);
                }
            }
    HE_TRY(dev_alloc(&F.Wm, wm.size()));
    HE_CHECK_CUDA(cudaMemcpy(F.Wm, wm.data(), wm.size() * 8, cudaMemcpyHostToDevice));
    return HE_OK;
}

static int factored_runtime(he_conv *cv) {
    he_ctx *c = cv->c;
    FactoredConv &F = *cv->fc;
    const size_t pw = cv->pw;
    HE_TRY(dev_alloc(&cv->R, (size_t)cv->lin.ns * 2 * pw));
    HE_TRY(dev_alloc(&F.Y, (size_t)F.nY * 2 * pw));
    HE_TRY(dev_alloc(&cv->acc, (size_t)cv->lout.ns * 2 * pw));
    HE_TRY(dev_alloc(&F.rt, (size_t)2 * std::max(F.nY, cv->lout.ns) * cv->level * c->n));
    if (cv->stride == 2) {
        HE_TRY(pool_build(c, cv->lout, cv->level - 2, true, &cv->pool));
        for (int v = 0; v < cv->lout.ns; v++) {
            he_ct *m;
            HE_TRY(he_ct_alloc(c, cv->level - 2, &m));
            cv->mid.push_back(m);
        }
    }
    return HE_OK;
}

static int factored_prepare(he_conv *cv, int mode) {
    he_ctx *c = cv->c;
    FactoredConv &F = *cv->fc;
    const size_t pw = cv->pw;
    const size_t pe = (size_t)(cv->level + 1 + c->K) * c->n;
    if (mode == HE_FUSED) {
        if (F.fy.c) return HE_OK;
        F.fy.c = c;
        F.fy.level = cv->level;
        char nm[96];
        snprintf(nm, sizeof(nm), "factored conv %d->%d %dx%d k%dx%d masks", cv->ci, cv->co, cv->lin.m, cv->lin.m,
                 cv->kh, cv->kw);
        F.fy.name = nm;
        for (int u = 0; u < cv->lin.ns; u++) F.fy.add_src(cv->R + (size_t)u * 2 * pw, pw);
        for (int y = 0; y < F.nY; y++) F.fy.add_out(F.Y + (size_t)y * 2 * pw, pw);
        for (int y = 0; y < F.nY; y++)
            for (int x = F.yoff[y]; x < F.yoff[y + 1]; x++) F.fy.add_term(y, F.ts[x], F.ta[x], F.masks + (size_t)F.tm[x] * pe);
        return F.fy.build();
    }
    if (F.rot_ready) return HE_OK;
    for (size_t x = 0; x < F.ts.size(); x++)
        if (F.ta[x] != 0) F.rslot.emplace(F.ts[x] * c->N + F.ta[x], (int)F.rslot.size());
    HE_TRY(dev_alloc(&F.Rrot, F.rslot.size() * 2 * pw));
    std::vector<mac_term> terms(F.ts.size());
    for (size_t x = 0; x < F.ts.size(); x++) {
        const u64 *src = F.ta[x] == 0 ? cv->R + (size_t)F.ts[x] * 2 * pw
                                      : F.Rrot + (size_t)F.rslot[F.ts[x] * c->N + F.ta[x]] * 2 * pw;
        terms[x] = mac_term{F.masks + (size_t)F.tm[x] * pe, src, pw};
    }
    HE_TRY(dev_alloc(&F.d_terms, std::max<size_t>(1, terms.size())));
    if (!terms.empty()) HE_CHECK_CUDA(cudaMemcpy(F.d_terms, terms.data(), terms.size() * sizeof(mac_term), cudaMemcpyHostToDevice));
    F.ry.c = c;
    F.ry.level = cv->level;
    for (int u = 0; u < cv->lin.ns; u++) F.ry.src.push_back({cv->R + (size_t)u * 2 * pw, pw});
    for (auto &kv : F.rslot) F.ry.add(kv.first / c->N, kv.first % c->N, F.Rrot + (size_t)kv.second * 2 * pw, pw);
    F.rot_ready = true;
    return HE_OK;
}

static int factored_run(he_ctx *c, he_conv *cv, he_ct *const *in, he_ct **out, int mode, cudaStream_t s) {
    FactoredConv &F = *cv->fc;
    const size_t pw = cv->pw;
    const int lv = cv->level;
    for (int u = 0; u < cv->lin.ns; u++) {
        if (!in[u] || in[u]->ctx != c || in[u]->level != lv || in[u]->scale != cv->in_scale) {
            he_set_error("he_conv_run: input shard %d is not at level %d / the planned scale", u, lv);
            return HE_ELEVEL;
        }
        HE_TRY(k_copy_limbs(cv->R + (size_t)u * 2 * pw, pw, in[u]->d, in[u]->pstride, pw, 2, s));
    }
    HE_TRY(factored_prepare(cv, mode));
    // stage 1: masked rotations, then one batched rescale of every Y
    if (mode == HE_FUSED) {
        HE_TRY(F.fy.run(s));
    } else {
        if (mode == HE_BATCHED) HE_TRY(F.ry.prepare_batched());
        HE_TRY(F.ry.run(mode, s));
        for (int y = 0; y < F.nY; y++)
            HE_TRY(k_mac(c, F.d_terms + F.yoff[y], F.yoff[y + 1] - F.yoff[y], F.Y + (size_t)y * 2 * pw, pw, lv, false, s));
    }
    HE_TRY(k_rescale_many(c, F.Y, pw, F.nY, lv, F.rt, s));
    const double y_scale = cv->in_scale * (double)c->primes[lv] / (double)c->primes[lv];
    // stage 2: integer scalars, rescale, bias
    const int l1 = lv - 1;
    HE_TRY(k_smac(c, F.Y, 2 * pw, pw, F.Wm, cv->co, cv->ci, F.H, F.T, l1, cv->acc, 2 * pw, pw, s));
    HE_TRY(k_rescale_many(c, cv->acc, pw, cv->lout.ns, l1, F.rt, s));
    const double o_scale = y_scale * (double)c->primes[l1] / (double)c->primes[l1];
    he_ct **dst = cv->stride == 1 ? out : cv->mid.data();
    for (int v = 0; v < cv->lout.ns; v++) {
        u64 *a = cv->acc + (size_t)v * 2 * pw;
        HE_TRY(k_add_raw(c, a, pw, cv->bias_pts + (size_t)v * (lv - 1) * c->n, 0, lv - 1, 1, false, s));
        if (!dst[v] || dst[v]->ctx != c) { he_set_error("he_conv_run: output %d missing", v); return HE_EINVAL; }
        HE_TRY(ensure_ct(c, dst[v], lv - 2));
        HE_TRY(k_copy_limbs(dst[v]->d, dst[v]->pstride, a, pw, (size_t)(lv - 1) * c->n, 2, s));
        dst[v]->scale = o_scale;
    }
    if (cv->stride == 2) {
        HE_TRY(pool_prepare(cv->pool, mode));
        return pool_run(c, cv->pool, cv->mid.data(), out, mode, s);
    }
    return HE_OK;
}

extern "C" int he_conv_create_factored(he_ctx *c, const he_layout *in, const double *W, const double *bias, int co,
                                       int ci, int kh, int kw, int stride, int pad, int level, double in_scale,
                                       he_conv **out) {
    if (!c || !in || !W || !out || co < 1 || ci < 1 || kh < 1 || kw < 1 || pad < 0 ||
        (stride != 1 && stride != 2)) {
        he_set_error("he_conv_create_factored: bad argument");
        return HE_EINVAL;
    }
    const int need = stride == 1 ? 2 : 4;
    if (level < need || level > c->L) { he_set_error("he_conv_create_factored: level %d leaves too few levels", level); return HE_ELEVEL; }
    Lay lin = from_c(*in);
    HE_TRY(check_layout(lin, c->N));
    if (lin.c != ci) { he_set_error("he_conv_create_factored: layout has %d channels, W has %d", lin.c, ci); return HE_EINVAL; }
    if (lin.nb != 1 || lin.B != lin.N || lin.ns != ci * (lin.M / lin.rows())) {
        he_set_error("he_conv_create_factored: the input must be in channel shards (each shard rows of one channel)");
        return HE_EINVAL;
    }
    for (int u = 0; u < lin.ns; u++)
        if (lin.chan[u] != u / (lin.M / lin.rows()) || lin.row0[u] != (u % (lin.M / lin.rows())) * lin.rows()) {
            he_set_error("he_conv_create_factored: shards must hold channels in order, rows in order");
            return HE_EINVAL;
        }
    std::unique_ptr<he_conv> cv(new he_conv());
    cv->c = c;
    cv->lin = lin;
    cv->lout = image_layout(co, lin.m, lin.N);
    cv->W.assign(W, W + (size_t)co * ci * kh * kw);
    if (bias) cv->bias.assign(bias, bias + co);
    cv->co = co; cv->ci = ci; cv->kh = kh; cv->kw = kw; cv->pad = pad; cv->stride = stride;
    cv->level = level;
    cv->in_scale = in_scale;
    cv->pw = (size_t)(level + 1) * c->n;
    cv->pe = (size_t)(level + 1 + c->K) * c->n;
    cv->fc.reset(new FactoredConv());
    FactoredConv &F = *cv->fc;
    std::vector<std::vector<double>> mvals;
    HE_TRY(factored_plan(cv.get(), mvals));
    HE_TRY(dev_alloc(&F.masks, (size_t)F.n_masks * cv->pe));
    std::vector<const double *> vecs;
    for (auto &v : mvals) vecs.push_back(v.data());
    HE_TRY(upload_plaintexts(c, vecs, vecs.size(), (double)c->primes[level], level, F.masks, nullptr, true));
    // bias at the output scale, normal NTT form at level - 2
    const double y_scale = in_scale * (double)c->primes[level] / (double)c->primes[level];
    const double o_scale = y_scale * (double)c->primes[level - 1] / (double)c->primes[level - 1];
    HE_TRY(dev_alloc(&cv->bias_pts, (size_t)cv->lout.ns * (level - 1) * c->n));
    for (int v = 0; v < cv->lout.ns; v++) {
        std::vector<int64_t> m;
        conv_bias_int(cv.get(), v, o_scale, m);
        HE_TRY(upload_addend(c, m.data(), level - 2, cv->bias_pts + (size_t)v * (level - 1) * c->n));
    }
    HE_TRY(factored_runtime(cv.get()));
    *out = cv.release();
    return HE_OK;
}


// buffers every mode uses: input copies, accumulators, the stride-2 select stage
// per-rotation BSGS: the giant rotations of every partial sum (amount 0: a copy)
static void bsgs_giant_set(he_conv *cv, RotSet &g, int level, size_t pw, u64 *Sb, u64 *Gb) {
    g.c = cv->c;
    g.level = level;
    for (size_t i = 0; i < cv->sv.size(); i++) g.src.push_back({Sb + i * 2 * pw, pw});
    for (size_t i = 0; i < cv->sv.size(); i++) g.add((int)i, cv->sg[i], Gb + i * 2 * pw, pw);
}

// per-rotation BSGS after the baby rotations: each partial sum's MAC (unrescaled), its giant
// rotation, and the sum of the rotated partial sums of every output shard into acc
static int bsgs_rot_tail(he_ctx *c, he_conv *cv, const mac_term *d_terms, u64 *Sb, u64 *Gb, u64 *acc, size_t pw,
                         int lv, RotSet &grot, int mode, cudaStream_t s) {
    const size_t nS = cv->sv.size();
    for (size_t i = 0; i < nS; i++)
        HE_TRY(k_mac(c, d_terms + cv->s_off[i], cv->s_off[i + 1] - cv->s_off[i], Sb + i * 2 * pw, pw, lv, false, s));
    if (mode == HE_BATCHED) HE_TRY(grot.prepare_batched());
    HE_TRY(grot.run(mode, s));
    std::vector<char> first(cv->lout.ns, 1);
    for (size_t i = 0; i < nS; i++) {
        const int v = cv->sv[i];
        u64 *a = acc + (size_t)v * 2 * pw;
        const u64 *x = Gb + i * 2 * pw;
        if (first[v]) HE_TRY(k_copy_limbs(a, pw, x, pw, pw, 2, s));
        else HE_TRY(k_add_raw(c, a, pw, x, pw, lv + 1, 2, false, s));
        first[v] = 0;
    }
    return HE_OK;
}

// fused BSGS stages of one image at level l: baby (inputs -> partial sums, one ModDown each)
// and giant (partial sums -> outputs, plaintext 1, one ModDown per output)
static int bsgs_fused_stages(he_conv *cv, FusedStage &B, FusedStage &G, int l, int pt_level, size_t pw, u64 *R,
                             u64 *Sb, u64 *acc, const std::string &name) {
    B.c = G.c = cv->c;
    B.level = G.level = l;
    B.pt_level = pt_level;
    B.name = name + " baby";
    G.name = name + " giant";
    for (int u = 0; u < cv->lin.ns; u++) B.add_src(R + (size_t)u * 2 * pw, pw);
    for (size_t i = 0; i < cv->sv.size(); i++) B.add_out(Sb + i * 2 * pw, pw);
    for (size_t t = 0; t < cv->tu.size(); t++) B.add_term(cv->ts[t], cv->tu[t], cv->tt[t], cv->pts + t * cv->pe);
    for (size_t i = 0; i < cv->sv.size(); i++) G.add_src(Sb + i * 2 * pw, pw);
    for (int v = 0; v < cv->lout.ns; v++) G.add_out(acc + (size_t)v * 2 * pw, pw);
    for (size_t i = 0; i < cv->sv.size(); i++) G.add_term(cv->sv[i], (int)i, cv->sg[i], HE_PT_ONE);
    HE_TRY(B.build());
    return G.build();
}

static int conv_runtime(he_conv *cv, const he_pool *pool_src = nullptr) {
    he_ctx *c = cv->c;
    HE_TRY(dev_alloc(&cv->R, (size_t)cv->lin.ns * 2 * cv->pw));
    HE_TRY(dev_alloc(&cv->acc, (size_t)cv->lout.ns * 2 * cv->pw));
    if (cv->bsgs) HE_TRY(dev_alloc(&cv->Sb, cv->sv.size() * 2 * cv->pw));
    if (cv->stride == 2) {
        if (pool_src) HE_TRY(pool_fork(pool_src, c, &cv->pool));
        else HE_TRY(pool_build(c, cv->lout, cv->level - 1, true, &cv->pool));
        for (int v = 0; v < cv->lout.ns; v++) {
            he_ct *m;
            HE_TRY(he_ct_alloc(c, cv->level - 1, &m));
            cv->mid.push_back(m);
        }
    }
    return HE_OK;
}

// rotation buffers, MAC tables and rotation set of the per-rotation modes
static int conv_rot_runtime(he_conv *cv) {
    if (cv->rot_ready) return HE_OK;
    he_ctx *c = cv->c;
    const size_t pw = cv->pw, n_terms = cv->tu.size();
    HE_TRY(dev_alloc(&cv->Rrot, cv->slot.size() * 2 * pw));
    std::vector<mac_term> terms(n_terms);
    for (size_t t = 0; t < n_terms; t++)
        terms[t] = mac_term{cv->pts + t * cv->pe, cv->rot_ptr(cv->tu[t], cv->term_amt(t)), pw};
    HE_TRY(dev_alloc(&cv->d_terms, n_terms));
    HE_CHECK_CUDA(cudaMemcpy(cv->d_terms, terms.data(), n_terms * sizeof(mac_term), cudaMemcpyHostToDevice));
    cv->rot.c = c;
    cv->rot.level = cv->level;
    for (int u = 0; u < cv->lin.ns; u++) cv->rot.src.push_back({cv->R + (size_t)u * 2 * pw, pw});
    for (auto &kv : cv->slot) {
        int u = (int)(kv.first / c->N), a = (int)(kv.first % c->N);
        cv->rot.add(u, a, cv->Rrot + (size_t)kv.second * 2 * pw, pw);
    }
    if (cv->bsgs) {
        HE_TRY(dev_alloc(&cv->Gb, cv->sv.size() * 2 * pw));
        bsgs_giant_set(cv, cv->grot, cv->level, pw, cv->Sb, cv->Gb);
    }
    cv->rot_ready = true;
    return HE_OK;
}

static int conv_fork(const he_conv *src, he_ctx *c, he_conv **out) {
    if (c->root() != src->c->root()) { he_set_error("fork: contexts do not share a root"); return HE_ESTATE; }
    if (src->fc) { he_set_error("fork: not available for the factored form"); return HE_EINVAL; }
    std::unique_ptr<he_conv> cv(new he_conv());
    cv->c = c;
    cv->lin = src->lin; cv->lout = src->lout; cv->W = src->W; cv->bias = src->bias;
    cv->co = src->co; cv->ci = src->ci; cv->kh = src->kh; cv->kw = src->kw; cv->pad = src->pad;
    cv->stride = src->stride; cv->level = src->level;
    cv->in_scale = src->in_scale; cv->mid_scale = src->mid_scale;
    cv->pw = src->pw; cv->pe = src->pe;
    cv->tu = src->tu; cv->tv = src->tv; cv->ta = src->ta; cv->term_off = src->term_off;
    cv->bsgs = src->bsgs;
    cv->bsgs_k = src->bsgs_k;
    cv->tt = src->tt; cv->ts = src->ts; cv->sv = src->sv; cv->sg = src->sg; cv->s_off = src->s_off;
    cv->slot = src->slot;
    cv->pts = src->pts;
    cv->bias_pts = src->bias_pts;
    cv->shared_pts = true;
    HE_TRY(conv_runtime(cv.get(), src->pool));
    *out = cv.release();
    return HE_OK;
}

extern "C" int he_conv_fork(const he_conv *src, he_ctx *ctx, he_conv **out) {
    if (!src || !ctx || !out) { he_set_error("he_conv_fork: null argument"); return HE_EINVAL; }
    return conv_fork(src, ctx, out);
}

extern "C" int he_pool_fork(const he_pool *src, he_ctx *ctx, he_pool **out) {
    if (!src || !ctx || !out) { he_set_error("he_pool_fork: null argument"); return HE_EINVAL; }
    return pool_fork(src, ctx, out);
}

// bsgs_k < 0: the diagonal form; 0: baby-step giant-step with the giant stride chosen by
// bsgs_cost; >= 1: with a giant stride of bsgs_k blocks
static int conv_create(he_ctx *c, const he_layout *in, const double *W, const double *bias, int co, int ci, int kh,
                       int kw, int stride, int pad, int level, double in_scale, int bsgs_k, he_conv **out) {
    const bool bsgs = bsgs_k >= 0;
    if (!c || !in || !W || !out || co < 1 || ci < 1 || kh < 1 || kw < 1 || pad < 0 ||
        (stride != 1 && stride != 2)) {
        he_set_error("he_conv_create: bad argument");
        return HE_EINVAL;
    }
    const int need = stride == 1 ? 1 : 3;
    if (level < need || level > c->L) { he_set_error("he_conv_create: level %d leaves too few levels", level); return HE_ELEVEL; }
    Lay lin = from_c(*in);
    HE_TRY(check_layout(lin, c->N));
    if (lin.c != ci) { he_set_error("he_conv_create: layout has %d channels, W has %d", lin.c, ci); return HE_EINVAL; }
    std::unique_ptr<he_conv> cv(new he_conv());
    cv->c = c;
    cv->lin = lin;
    cv->lout = image_layout(co, lin.m, lin.N);
    if (cv->lout.M != lin.M) { he_set_error("he_conv_create: output frame differs"); return HE_EINVAL; }
    if ((size_t)cv->lout.ns * cv->lout.nb > HE_MAX_BLOCKS) { he_set_error("output layout too large"); return HE_EINVAL; }
    cv->W.assign(W, W + (size_t)co * ci * kh * kw);
    if (bias) cv->bias.assign(bias, bias + co);
    cv->co = co; cv->ci = ci; cv->kh = kh; cv->kw = kw; cv->pad = pad; cv->stride = stride;
    cv->level = level;
    cv->in_scale = in_scale;
    cv->mid_scale = in_scale * (double)c->primes[level] / (double)c->primes[level];
    cv->pw = (size_t)(level + 1) * c->n;
    cv->pe = (size_t)(level + 1 + c->K) * c->n;
    const size_t pw = cv->pw, pe = cv->pe;
    // plan all output shards, keeping the diagonals of one shard at a time
    std::vector<DiagMap> maps(cv->lout.ns);
    size_t n_terms = 0;
    for (int v = 0; v < cv->lout.ns; v++) {
        plan_conv_v(lin, cv->lout, cv->W.data(), ci, kh, kw, pad, v, maps[v]);
        n_terms += maps[v].size();
    }
    const int N = c->N;
    cv->bsgs = bsgs;
    if (bsgs) {
        if (bsgs_k > 0 && (bsgs_k > lin.nb || lin.nb % bsgs_k != 0 || (bsgs_k & (bsgs_k - 1)) != 0)) {
            he_set_error("he_conv_create_bsgs: giant stride %d blocks does not divide the %d blocks of a shard",
                         bsgs_k, lin.nb);
            return HE_EINVAL;
        }
        if (bsgs_k == 0) {                     // the modelled-fastest giant stride
            std::vector<std::array<int, 3>> tl;
            for (int v = 0; v < cv->lout.ns; v++)
                for (auto &kv : maps[v]) tl.push_back({v, (int)(kv.first / N), (int)(kv.first % N)});
            std::string note = "conv " + std::to_string(ci) + "->" + std::to_string(co) + " " + std::to_string(lin.m) +
                               "x" + std::to_string(lin.m) + " bsgs giant stride:";
            double best = 0;
            for (int k = 1; k <= lin.nb; k *= 2) {
                const double t = bsgs_cost(c, lin, level, tl, cv->lout.ns, k);
                char b[48];
                snprintf(b, sizeof(b), " k=%d %.0f us;", k, t);
                note += b;
                if (bsgs_k == 0 || t < best) { best = t; bsgs_k = k; }
            }
            he_tune_note(c, note + " -> k=" + std::to_string(bsgs_k));
        }
        cv->bsgs_k = bsgs_k;
    }
    // rotation slots: every (u, amount) with amount != 0 that some term's input needs (the
    // diagonal amount a, or in the BSGS form the baby amount t)
    for (int v = 0; v < cv->lout.ns; v++)
        for (auto &kv : maps[v]) {
            int a = (int)(kv.first % N), g = 0, t = a;
            if (bsgs) bsgs_split(a, lin.B, N, bsgs_k, g, t);
            const long long key = (kv.first / N) * N + t;
            if (t != 0 && !cv->slot.count(key)) {
                int id = (int)cv->slot.size();
                cv->slot[key] = id;
            }
        }
    HE_TRY(dev_alloc(&cv->pts, n_terms * pe));
    HE_TRY(dev_alloc(&cv->bias_pts, (size_t)cv->lout.ns * level * c->n));
    // diagonal plaintexts at scale q_level; in the BSGS form ordered by (g, u, t) within an
    // output shard, the diagonal rotated by -g: P'[i] = D[(i - g) mod N]
    size_t t0 = 0;
    cv->term_off.push_back(0);
    for (int v = 0; v < cv->lout.ns; v++) {
        struct E { int g, u, t, a; const std::vector<double> *D; };
        std::vector<E> es;
        for (auto &kv : maps[v]) {
            int a = (int)(kv.first % N), g = 0, t = a;
            if (bsgs) bsgs_split(a, lin.B, N, bsgs_k, g, t);
            es.push_back({g, (int)(kv.first / N), t, a, &kv.second});
        }
        if (bsgs)
            std::sort(es.begin(), es.end(), [](const E &x, const E &y) {
                return x.g != y.g ? x.g < y.g : x.u != y.u ? x.u < y.u : x.t < y.t;
            });
        std::vector<std::vector<double>> rolled;
        std::vector<const double *> vecs;
        if (bsgs) rolled.reserve(es.size());
        for (const E &e : es) {
            cv->tu.push_back(e.u);
            cv->tv.push_back(v);
            cv->ta.push_back(e.a);
            if (bsgs) {
                if (cv->sv.empty() || cv->sv.back() != v || cv->sg.back() != e.g) {
                    cv->sv.push_back(v);
                    cv->sg.push_back(e.g);
                    cv->s_off.push_back((int)cv->tu.size() - 1);
                }
                cv->tt.push_back(e.t);
                cv->ts.push_back((int)cv->sv.size() - 1);
                std::vector<double> r(N);
                for (int i = 0; i < N; i++) r[i] = (*e.D)[((i - e.g) % N + N) % N];
                rolled.push_back(std::move(r));
                vecs.push_back(rolled.back().data());
            } else {
                vecs.push_back(e.D->data());
            }
        }
        HE_TRY(upload_plaintexts(c, vecs, vecs.size(), (double)c->primes[level], level, cv->pts + t0 * pe, nullptr,
                                 true));
        t0 += vecs.size();
        cv->term_off.push_back((int)t0);
        DiagMap().swap(maps[v]);
    }
    if (bsgs) cv->s_off.push_back((int)t0);
    // bias at the output scale, normal NTT form at level - 1
    for (int v = 0; v < cv->lout.ns; v++) {
        std::vector<int64_t> m;
        conv_bias_int(cv.get(), v, cv->mid_scale, m);
        HE_TRY(upload_addend(c, m.data(), level - 1, cv->bias_pts + (size_t)v * level * c->n));
    }
    HE_TRY(conv_runtime(cv.get()));
    *out = cv.release();
    return HE_OK;
}

extern "C" int he_conv_create(he_ctx *c, const he_layout *in, const double *W, const double *bias,
                              int co, int ci, int kh, int kw, int stride, int pad, int level,
                              double in_scale, he_conv **out) {
    return conv_create(c, in, W, bias, co, ci, kh, kw, stride, pad, level, in_scale, -1, out);
}

extern "C" int he_conv_create_bsgs(he_ctx *c, const he_layout *in, const double *W, const double *bias,
                                   int co, int ci, int kh, int kw, int stride, int pad, int level,
                                   double in_scale, int giant_blocks, he_conv **out) {
    if (giant_blocks < 0) { he_set_error("he_conv_create_bsgs: negative giant stride"); return HE_EINVAL; }
    return conv_create(c, in, W, bias, co, ci, kh, kw, stride, pad, level, in_scale, giant_blocks, out);
}

extern "C" int he_conv_bsgs_giant(const he_conv *cv) {
    if (!cv) return HE_EINVAL;
    return cv->bsgs ? cv->bsgs_k : 0;
}

extern "C" void he_conv_destroy(he_conv *cv) {
    if (cv) { cudaDeviceSynchronize(); delete cv; }
}
extern "C" int he_conv_out_layout(const he_conv *cv, he_layout *out) {
    if (!cv || !out) return HE_EINVAL;
    return to_c(cv->pool ? cv->pool->P.lout : cv->lout, out);
}
extern "C" int he_conv_select_pool(const he_conv *cv, he_pool **out) {
    if (!cv || !out) { he_set_error("he_conv_select_pool: null argument"); return HE_EINVAL; }
    *out = nullptr;
    if (cv->stride != 2 || !cv->pool) {
        he_set_error("he_conv_select_pool: only a stride-2 convolution has a select stage");
        return HE_EINVAL;
    }
    *out = cv->pool;
    return HE_OK;
}
extern "C" int he_conv_out_level(const he_conv *cv) {
    if (!cv) return HE_EINVAL;
    if (cv->fc) return cv->stride == 1 ? cv->level - 2 : cv->level - 4;
    return cv->stride == 1 ? cv->level - 1 : cv->level - 3;
}
extern "C" int he_conv_rotations(const he_conv *cv, int32_t *amounts, size_t cap) {
    if (!cv) return HE_EINVAL;
    std::vector<int> v;
    for (auto &kv : cv->slot) v.push_back((int)(kv.first % cv->c->N));
    v.insert(v.end(), cv->sg.begin(), cv->sg.end());
    if (cv->fc) v.insert(v.end(), cv->fc->amt.begin(), cv->fc->amt.end());
    if (cv->pool) collect_rotations(cv->pool, v);
    return distinct_nonzero(cv->c, v, amounts, cap);
}
// key switches one run performs: distinct (source, nonzero amount) pairs of every stage
static int64_t pool_keyswitches(const he_pool *p) {
    const PoolPlanH &P = p->P;
    he_ctx *c = p->c;
    auto nz = [&](int a) { return h_galois(c, a) != 1; };
    int64_t k = 0;
    for (int a : P.pre) k += nz(a) ? p->ns : 0;
    for (int a : P.h_amt) k += nz(a) ? p->ns : 0;
    for (int a : P.v_amt) k += nz(a) ? p->ns : 0;
    std::set<std::pair<int, int>> cs;
    for (auto &g : P.groups)
        for (auto &ua : g)
            if (nz(ua.second)) cs.insert(ua);
    k += (int64_t)cs.size();
    for (int a : P.dup)
        if (nz(a)) k += (int64_t)P.groups.size();
    return k;
}

extern "C" int64_t he_pool_keyswitches(const he_pool *p) { return p ? pool_keyswitches(p) : HE_EINVAL; }

extern "C" int64_t he_conv_keyswitches(const he_conv *cv) {
    if (!cv) return HE_EINVAL;
    int64_t k = 0;
    if (cv->fc) {
        std::set<std::pair<int, int>> r;
        for (size_t x = 0; x < cv->fc->ts.size(); x++)
            if (h_galois(cv->c, cv->fc->ta[x]) != 1) r.insert({cv->fc->ts[x], cv->fc->ta[x]});
        k = (int64_t)r.size();
    } else {
        k = (int64_t)cv->slot.size();
        for (int g : cv->sg) k += h_galois(cv->c, g) != 1;
    }
    if (cv->pool) k += pool_keyswitches(cv->pool);
    return k;
}

extern "C" int he_conv_n_terms(const he_conv *cv) {
    if (!cv) return HE_EINVAL;
    return cv->fc ? cv->fc->n_masks : (int)cv->tu.size();
}

extern "C" int he_conv_export_plan(const he_conv *cv, int32_t *u, int32_t *v, int32_t *a, double *diag) {
    if (!cv) return HE_EINVAL;
    if (cv->fc) {                               // masks: u = source shard h', v = shard h, a = a_t
        std::vector<std::array<int, 3>> keys;
        std::vector<std::vector<double>> mv;
        std::vector<int> amt;
        HE_TRY(factored_masks(cv, keys, mv, amt));
        for (size_t m = 0; m < keys.size(); m++) {
            if (u) u[m] = keys[m][1];
            if (v) v[m] = keys[m][0];
            if (a) a[m] = amt[keys[m][2]];
            if (diag) memcpy(diag + m * (size_t)cv->c->N, mv[m].data(), (size_t)cv->c->N * 8);
        }
        return HE_OK;
    }
    for (size_t t = 0; t < cv->tu.size(); t++) {
        if (u) u[t] = cv->tu[t];
        if (v) v[t] = cv->tv[t];
        if (a) a[t] = cv->ta[t];
    }
    if (diag) {                                 // the diagonal D_{u,v,a} of every term
        const int N = cv->c->N;
        for (int vv = 0; vv < cv->lout.ns; vv++) {
            DiagMap m;
            plan_conv_v(cv->lin, cv->lout, cv->W.data(), cv->ci, cv->kh, cv->kw, cv->pad, vv, m);
            for (int t = cv->term_off[vv]; t < cv->term_off[vv + 1]; t++)
                memcpy(diag + (size_t)t * N, m[(long long)cv->tu[t] * N + cv->ta[t]].data(), (size_t)N * 8);
        }
    }
    return HE_OK;
}

static void conv_invalidate_pk(he_conv *cv);

extern "C" int he_conv_import_plaintexts(he_conv *cv, const int64_t *terms, const int64_t *bias) {
    if (!cv) return HE_EINVAL;
    he_ctx *c = cv->c;
    if (cv->fc) {                               // masks [n_masks][n] at scale q_l, bias at l - 2
        std::vector<const double *> none;
        if (terms) HE_TRY(upload_plaintexts(c, none, cv->fc->n_masks, 0.0, cv->level, cv->fc->masks, terms, true));
        if (bias)
            for (int v = 0; v < cv->lout.ns; v++)
                HE_TRY(upload_addend(c, bias + (size_t)v * c->n, cv->level - 2,
                                     cv->bias_pts + (size_t)v * (cv->level - 1) * c->n));
        if (terms) conv_invalidate_pk(cv);
        return HE_OK;
    }
    if (terms) {
        std::vector<const double *> none;
        HE_TRY(upload_plaintexts(c, none, cv->tu.size(), 0.0, cv->level, cv->pts, terms, true));
        conv_invalidate_pk(cv);
    }
    if (bias)
        for (int v = 0; v < cv->lout.ns; v++)
            HE_TRY(upload_addend(c, bias + (size_t)v * c->n, cv->level - 1, cv->bias_pts + (size_t)v * cv->level * c->n));
    return HE_OK;
}

static int conv_prepare_fused(he_conv *cv) {
    FusedStage &F = cv->fused;
    if (F.c) return HE_OK;
    char nm[96];
    snprintf(nm, sizeof(nm), "conv %d->%d %dx%d k%dx%d", cv->ci, cv->co, cv->lin.m, cv->lin.m, cv->kh, cv->kw);
    if (cv->bsgs) return bsgs_fused_stages(cv, F, cv->fusedG, cv->level, cv->level, cv->pw, cv->R, cv->Sb, cv->acc, nm);
    F.c = cv->c;
    F.level = cv->level;
    F.name = nm;
    for (int u = 0; u < cv->lin.ns; u++) F.add_src(cv->R + (size_t)u * 2 * cv->pw, cv->pw);
    for (int v = 0; v < cv->lout.ns; v++) F.add_out(cv->acc + (size_t)v * 2 * cv->pw, cv->pw);
    for (size_t t = 0; t < cv->tu.size(); t++) F.add_term(cv->tv[t], cv->tu[t], cv->ta[t], cv->pts + t * cv->pe);
    return F.build();
}

static int factored_run(he_ctx *c, he_conv *cv, he_ct *const *in, he_ct **out, int mode, cudaStream_t s);

extern "C" int he_conv_run(he_ctx *c, he_conv *cv, he_ct *const *in, he_ct **out, int mode, void *stream) {
    if (!c || !cv || !in || !out || cv->c != c || (mode != HE_PLAIN && mode != HE_BATCHED && mode != HE_FUSED)) {
        he_set_error("he_conv_run: bad argument");
        return HE_EINVAL;
    }
    if (cv->fc) return factored_run(c, cv, in, out, mode, (cudaStream_t)stream);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t pw = cv->pw;
    const int lv = cv->level;
    for (int u = 0; u < cv->lin.ns; u++) {
        if (!in[u] || in[u]->ctx != c || in[u]->level != lv || in[u]->scale != cv->in_scale) {
            he_set_error("he_conv_run: input shard %d is not at level %d / the planned scale", u, lv);
            return HE_ELEVEL;
        }
        HE_TRY(k_copy_limbs(cv->R + (size_t)u * 2 * pw, pw, in[u]->d, in[u]->pstride, pw, 2, s));
    }
    if (mode == HE_FUSED) {
        HE_TRY(conv_prepare_fused(cv));
        HE_TRY(cv->fused.run(s));
        if (cv->bsgs) HE_TRY(cv->fusedG.run(s));
    } else {
        HE_TRY(conv_rot_runtime(cv));
        if (mode == HE_BATCHED) HE_TRY(cv->rot.prepare_batched());
        HE_TRY(cv->rot.run(mode, s));
        if (cv->bsgs) HE_TRY(bsgs_rot_tail(c, cv, cv->d_terms, cv->Sb, cv->Gb, cv->acc, pw, lv, cv->grot, mode, s));
    }
    he_ct **dst = cv->stride == 1 ? out : cv->mid.data();
    for (int v = 0; v < cv->lout.ns; v++) {
        // MAC over all (u, a) terms of output shard v (fused mode: already in acc), rescale,
        // add the bias, hand out
        u64 *a = cv->acc + (size_t)v * 2 * pw;
        const int t0 = cv->term_off[v], t1 = cv->term_off[v + 1];
        if (mode != HE_FUSED && !cv->bsgs) HE_TRY(k_mac(c, cv->d_terms + t0, t1 - t0, a, pw, lv, false, s));
        he_ct t = view(c, a, pw, lv, cv->in_scale * (double)c->primes[lv]);
        HE_TRY(he_rescale(c, &t, stream));
        HE_TRY(k_add_raw(c, a, pw, cv->bias_pts + (size_t)v * lv * c->n, 0, lv, 1, false, s));
        if (!dst[v] || dst[v]->ctx != c) { he_set_error("he_conv_run: output %d missing", v); return HE_EINVAL; }
        HE_TRY(ensure_ct(c, dst[v], lv - 1));
        HE_TRY(k_copy_limbs(dst[v]->d, dst[v]->pstride, a, pw, (size_t)lv * c->n, 2, s));
        dst[v]->scale = t.scale;
    }
    if (cv->stride == 2) {
        HE_TRY(pool_prepare(cv->pool, mode));
        return pool_run(c, cv->pool, cv->mid.data(), out, mode, s);
    }
    return HE_OK;
}

// ================================================================================ image batches
// Several images through one convolution, each at its own level l_i <= the layer's level
// (the plaintexts, encoded once for the layer's level, serve every lower level: an integer
// plaintext's residues mod q_0..q_l and P are a subset of the stored ones).  In HE_FUSED mode
// every image's rotations, inner products and MACs run in ONE fused-kernel launch whose groups
// span all images and levels; the per-rotation modes run image by image.
struct ConvSlot {                                // one image of a batch: buffers at its level
    int level = 0;
    size_t pw = 0;
    u64 *R = nullptr, *acc = nullptr, *Rrot = nullptr;
    u64 *Sb = nullptr, *Gb = nullptr;            // BSGS partial sums, rotated partial sums
    mac_term *d_terms = nullptr;
    RotSet rot, grot;
    bool rot_ready = false;
    FusedStage fused, fusedG;                    // fusedG: BSGS giant stage
    ~ConvSlot() { he_free(R); he_free(acc); he_free(Rrot); he_free(d_terms); he_free(Sb); he_free(Gb); }
};
struct ConvBatch {
    std::vector<int> levels;
    std::vector<std::unique_ptr<ConvSlot>> slots;
    std::unique_ptr<FusedLaunch> launch, launchG;   // launchG: the BSGS giant stages
};

he_conv::~he_conv() {
    batch.reset();
    fc.reset();
    for (auto &kv : bias_by) he_free(kv.second);
    he_free(R); he_free(Rrot); he_free(d_terms); he_free(acc); he_free(Sb); he_free(Gb);
    if (!shared_pts) { he_free(pts); he_free(bias_pts); }
    delete pool;
    for (he_ct *x : mid) he_ct_free(x);
}

static int conv_batch_build(he_conv *cv, const std::vector<int> &levels) {
    he_ctx *c = cv->c;
    HE_TRY(he_capture_guard("a new batch signature"));
    std::unique_ptr<ConvBatch> B(new ConvBatch());
    B->levels = levels;
    B->launch.reset(new FusedLaunch());
    B->launch->c = c;
    char nm[128];
    snprintf(nm, sizeof(nm), "conv %d->%d %dx%d k%dx%d batch of %zu", cv->ci, cv->co, cv->lin.m, cv->lin.m, cv->kh,
             cv->kw, levels.size());
    B->launch->name = nm;
    if (cv->bsgs) {
        B->launchG.reset(new FusedLaunch());
        B->launchG->c = c;
        B->launchG->name = std::string(nm) + " giant";
        B->launch->name += " baby";
    }
    for (size_t i = 0; i < levels.size(); i++) {
        std::unique_ptr<ConvSlot> S(new ConvSlot());
        const int l = levels[i];
        S->level = l;
        S->pw = (size_t)(l + 1) * c->n;
        HE_TRY(dev_alloc(&S->R, (size_t)cv->lin.ns * 2 * S->pw));
        HE_TRY(dev_alloc(&S->acc, (size_t)cv->lout.ns * 2 * S->pw));
        if (cv->bsgs) {
            HE_TRY(dev_alloc(&S->Sb, cv->sv.size() * 2 * S->pw));
            HE_TRY(bsgs_fused_stages(cv, S->fused, S->fusedG, l, cv->level, S->pw, S->R, S->Sb, S->acc,
                                     std::string(nm) + " image " + std::to_string(i)));
            B->launch->st.push_back(&S->fused);
            B->launchG->st.push_back(&S->fusedG);
            B->slots.push_back(std::move(S));
            continue;
        }
        FusedStage &F = S->fused;
        F.c = c;
        F.level = l;
        F.pt_level = cv->level;
        F.name = std::string(nm) + " image " + std::to_string(i);
        for (int u = 0; u < cv->lin.ns; u++) F.add_src(S->R + (size_t)u * 2 * S->pw, S->pw);
        for (int v = 0; v < cv->lout.ns; v++) F.add_out(S->acc + (size_t)v * 2 * S->pw, S->pw);
        for (size_t t = 0; t < cv->tu.size(); t++) F.add_term(cv->tv[t], cv->tu[t], cv->ta[t], cv->pts + t * cv->pe);
        HE_TRY(F.build());
        B->launch->st.push_back(&F);
        B->slots.push_back(std::move(S));
    }
    cv->batch.reset(B.release());
    return HE_OK;
}

// rotation buffers and MAC tables of one image for the per-rotation modes
static int conv_slot_rot(he_conv *cv, ConvSlot &S) {
    if (S.rot_ready) return HE_OK;
    he_ctx *c = cv->c;
    const size_t pw = S.pw, n_terms = cv->tu.size();
    std::map<long long, int> slot = cv->slot;
    HE_TRY(dev_alloc(&S.Rrot, slot.size() * 2 * pw));
    auto rptr = [&](int u, int a) {
        return a == 0 ? S.R + (size_t)u * 2 * pw : S.Rrot + (size_t)slot[(long long)u * c->N + a] * 2 * pw;
    };
    std::vector<mac_term> terms(n_terms);
    for (size_t t = 0; t < n_terms; t++) terms[t] = mac_term{cv->pts + t * cv->pe, rptr(cv->tu[t], cv->term_amt(t)), pw};
    HE_TRY(dev_alloc(&S.d_terms, n_terms));
    HE_CHECK_CUDA(cudaMemcpy(S.d_terms, terms.data(), n_terms * sizeof(mac_term), cudaMemcpyHostToDevice));
    S.rot.c = c;
    S.rot.level = S.level;
    for (int u = 0; u < cv->lin.ns; u++) S.rot.src.push_back({S.R + (size_t)u * 2 * pw, pw});
    for (auto &kv : slot) {
        int u = (int)(kv.first / c->N), a = (int)(kv.first % c->N);
        S.rot.add(u, a, S.Rrot + (size_t)kv.second * 2 * pw, pw);
    }
    if (cv->bsgs) {
        HE_TRY(dev_alloc(&S.Gb, cv->sv.size() * 2 * pw));
        bsgs_giant_set(cv, S.grot, S.level, pw, S.Sb, S.Gb);
    }
    S.rot_ready = true;
    return HE_OK;
}

static uint64_t scale_bits(double x) {
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
}

// bias addends [n_out][l][n] at level l - 1 and the given output scale (encoded on first use)
static int conv_bias_for(he_conv *cv, int l, double out_scale, const u64 **out) {
    auto key = std::make_pair(l, scale_bits(out_scale));
    auto it = cv->bias_by.find(key);
    if (it == cv->bias_by.end()) {
        HE_TRY(he_capture_guard("bias encoding for a new level or scale"));
        u64 *d;
        HE_TRY(dev_alloc(&d, (size_t)cv->lout.ns * l * cv->c->n));
        for (int v = 0; v < cv->lout.ns; v++) {
            std::vector<int64_t> m;
            conv_bias_int(cv, v, out_scale, m);
            int rc = upload_addend(cv->c, m.data(), l - 1, d + (size_t)v * l * cv->c->n);
            if (rc != HE_OK) { he_free(d); return rc; }
        }
        it = cv->bias_by.emplace(key, d).first;
    }
    *out = it->second;
    return HE_OK;
}

extern "C" int he_conv_import_bias(he_conv *cv, int level, double out_scale, const int64_t *bias) {
    if (!cv || !bias || level < 1 || level > cv->level) { he_set_error("he_conv_import_bias: bad argument"); return HE_EINVAL; }
    auto key = std::make_pair(level, scale_bits(out_scale));
    auto it = cv->bias_by.find(key);
    u64 *d;
    if (it != cv->bias_by.end()) d = it->second;
    else {
        HE_TRY(dev_alloc(&d, (size_t)cv->lout.ns * level * cv->c->n));
        cv->bias_by.emplace(key, d);
    }
    for (int v = 0; v < cv->lout.ns; v++)
        HE_TRY(upload_addend(cv->c, bias + (size_t)v * cv->c->n, level - 1, d + (size_t)v * level * cv->c->n));
    return HE_OK;
}

// new plaintext contents: every stage of this convolution (single run, image batch, factored
// stage 1) drops its pre-keyed tables
static void conv_invalidate_pk(he_conv *cv) {
    cv->fused.invalidate_pk();
    cv->fusedG.invalidate_pk();
    if (cv->fc) cv->fc->fy.invalidate_pk();
    if (cv->batch) {
        for (auto &S : cv->batch->slots) {
            S->fused.invalidate_pk();
            S->fusedG.invalidate_pk();
        }
        if (cv->batch->launch) cv->batch->launch->reset_pk();
        if (cv->batch->launchG) cv->batch->launchG->reset_pk();
    }
}

extern "C" int he_conv_run_batch(he_ctx *c, he_conv *cv, he_ct *const *in, he_ct **out, int n_img, int mode,
                                 void *stream) {
    if (!c || !cv || !in || !out || cv->c != c || n_img < 1 ||
        (mode != HE_PLAIN && mode != HE_BATCHED && mode != HE_FUSED)) {
        he_set_error("he_conv_run_batch: bad argument");
        return HE_EINVAL;
    }
    if (cv->stride != 1 || cv->fc) { he_set_error("he_conv_run_batch: stride-1 diagonal convolutions only"); return HE_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const int ni = cv->lin.ns, no = cv->lout.ns;
    std::vector<int> levels(n_img);
    for (int i = 0; i < n_img; i++) {
        const he_ct *x0 = in[(size_t)i * ni];
        if (!x0 || x0->ctx != c) { he_set_error("he_conv_run_batch: image %d input missing", i); return HE_EINVAL; }
        levels[i] = x0->level;
        if (levels[i] < 1 || levels[i] > cv->level) {
            he_set_error("he_conv_run_batch: image %d at level %d, the layer takes 1..%d", i, levels[i], cv->level);
            return HE_ELEVEL;
        }
        for (int u = 0; u < ni; u++) {
            const he_ct *x = in[(size_t)i * ni + u];
            if (!x || x->ctx != c || x->level != levels[i] || x->scale != x0->scale) {
                he_set_error("he_conv_run_batch: image %d shard %d differs in level or scale", i, u);
                return HE_ELEVEL;
            }
        }
    }
    if (!cv->batch || cv->batch->levels != levels) HE_TRY(conv_batch_build(cv, levels));
    ConvBatch &B = *cv->batch;
    for (int i = 0; i < n_img; i++) {
        ConvSlot &S = *B.slots[i];
        for (int u = 0; u < ni; u++) {
            const he_ct *x = in[(size_t)i * ni + u];
            HE_TRY(k_copy_limbs(S.R + (size_t)u * 2 * S.pw, S.pw, x->d, x->pstride, S.pw, 2, s));
        }
    }
    if (mode == HE_FUSED) {
        HE_TRY(B.launch->run(s));
        if (B.launchG) HE_TRY(B.launchG->run(s));
    } else {
        for (int i = 0; i < n_img; i++) {
            ConvSlot &S = *B.slots[i];
            HE_TRY(conv_slot_rot(cv, S));
            if (mode == HE_BATCHED) HE_TRY(S.rot.prepare_batched());
            HE_TRY(S.rot.run(mode, s));
            if (cv->bsgs) HE_TRY(bsgs_rot_tail(c, cv, S.d_terms, S.Sb, S.Gb, S.acc, S.pw, S.level, S.grot, mode, s));
        }
    }
    const double S_pt = (double)c->primes[cv->level];
    for (int i = 0; i < n_img; i++) {
        ConvSlot &S = *B.slots[i];
        const int l = S.level;
        const double in_scale = in[(size_t)i * ni]->scale;
        const double out_scale = in_scale * S_pt / (double)c->primes[l];
        const u64 *bias;
        HE_TRY(conv_bias_for(cv, l, out_scale, &bias));
        for (int v = 0; v < no; v++) {
            u64 *a = S.acc + (size_t)v * 2 * S.pw;
            const int t0 = cv->term_off[v], t1 = cv->term_off[v + 1];
            if (mode != HE_FUSED && !cv->bsgs) HE_TRY(k_mac(c, S.d_terms + t0, t1 - t0, a, S.pw, l, false, s));
            he_ct t = view(c, a, S.pw, l, in_scale * S_pt);
            HE_TRY(he_rescale(c, &t, stream));
            HE_TRY(k_add_raw(c, a, S.pw, bias + (size_t)v * l * c->n, 0, l, 1, false, s));
            he_ct *d = out[(size_t)i * no + v];
            if (!d || d->ctx != c) { he_set_error("he_conv_run_batch: output %d of image %d missing", v, i); return HE_EINVAL; }
            HE_TRY(ensure_ct(c, d, l - 1));
            HE_TRY(k_copy_limbs(d->d, d->pstride, a, S.pw, (size_t)l * c->n, 2, s));
            d->scale = t.scale;
        }
    }
    return HE_OK;
}

// ================================================================================ polynomial
// Relinearised products of several ciphertext pairs at one level in one set of launches per
// kernel: tensor, ModUp of every d2, one inner-product launch with the relinearisation key
// (read once per launch for all pairs), one ModDown pipeline, then the rescales.  Each
// product gets exactly the bits he_mul_relin gives it.
static int relin_batch(he_ctx *c, const std::vector<const he_ct *> &A, const std::vector<const he_ct *> &B,
                       const std::vector<he_ct *> &out, cudaStream_t s) {
    const int m = (int)A.size();
    if (m == 0) return HE_OK;
    const int l = A[0]->level;
    for (int i = 0; i < m; i++)
        if (A[i]->level != l || B[i]->level != l) { he_set_error("relin_batch: levels differ"); return HE_ELEVEL; }
    if (l < 1) { he_set_error("relin_batch: no level left"); return HE_ELEVEL; }
    const DeviceKey *key;
    HE_TRY(get_key(c, 0, &key));
    const int nq = l + 1, ext = nq + c->K, beta = (l + c->alpha) / c->alpha;
    const size_t n = c->n, wq = (size_t)nq * n, we = (size_t)ext * n;
    const size_t per = 3 * wq + wq + (size_t)beta * we + 2 * we + 2 * wq + 2 * wq;
    HE_TRY(c->sc_relin.ensure((size_t)m * per));
    u64 *d = c->sc_relin.p;                       // [m][3][nq][n]
    u64 *xc = d + (size_t)m * 3 * wq;             // [m][nq][n]
    u64 *D = xc + (size_t)m * wq;                 // [m][beta][ext][n]
    u64 *u = D + (size_t)m * beta * we;           // [m][2][ext][n]
    u64 *conv = u + (size_t)m * 2 * we;           // [m][2][nq][n] (the fused ModDown-rescale's w)
    HE_TRY(k_tensor_batch(c, A.data(), B.data(), m, d, 3 * wq, l, s));
    HE_TRY(k_copy_limbs(xc, wq, d + 2 * wq, 3 * wq, wq, m, s));
    ntt_job ji{xc, wq, 0, nq, nq, 0, m, 0};
    HE_TRY(k_ntt(c, ji, true, s));
    HE_TRY(k_modup_strided(c, xc, wq, d + 2 * wq, 3 * wq, D, (size_t)beta * we, m, l, s));
    ntt_job jd{D, we, 0, ext, nq, c->alpha, beta * m, beta};
    HE_TRY(k_ntt(c, jd, false, s));
    std::vector<ip_item> ip(m);
    for (int i = 0; i < m; i++) {
        HE_TRY(ensure_ct(c, out[i], l));
        ip[i] = ip_item{D + (size_t)i * beta * we, key->d, u + (size_t)i * 2 * we, 1, beta};
    }
    HE_TRY(k_inner_product_inline(c, ip.data(), m, l, s));
    // ModDown fused with the rescale: the bits of ModDown, then rescale
    std::vector<u64 *> op(m);
    std::vector<size_t> ops(m);
    for (int i = 0; i < m; i++) { op[i] = out[i]->d; ops[i] = out[i]->pstride; }
    HE_TRY(k_moddown_rescale(c, u, d, 3 * wq, wq, conv, op.data(), ops.data(), m, l, s));
    for (int i = 0; i < m; i++) {
        out[i]->scale = A[i]->scale * B[i]->scale;
        out[i]->level = l - 1;
        out[i]->scale = out[i]->scale / (double)c->primes[l];
    }
    return HE_OK;
}

// sum_k c_k T_k(x): T_{2k} = 2 T_k^2 - 1, T_{2k+1} = 2 T_k T_{k+1} - T_1 (Appendix), then the
// linear combination with exact-scale integer constants round(c S_t q_l / s) at the lowest
// level, the constant term round(c_0 S_t q_l) on coefficient 0, and one rescale.  All T_k of
// one tree depth read operands of lower depth at one common level, so each depth is one
// batched relinearisation.
static int retarget(he_ctx *c, const he_ct *x, int level, double scale_t, he_ct *y, cudaStream_t s) {
    HE_TRY(he_ct_copy(y, x, s));
    HE_TRY(he_ct_drop_level(y, level + 1));
    double K = std::nearbyint(scale_t * (double)c->primes[level + 1] / y->scale);
    HE_TRY(he_mul_int(c, y, K, s));
    HE_TRY(he_rescale(c, y, s));
    y->scale = scale_t;
    return HE_OK;
}

// Temporaries of the polynomial evaluator: `need` ciphertexts at level L in one allocation,
// kept in the context and reused by every call.
static int poly_temps(he_ctx *c, size_t need) {
    if (c->poly_tmp.size() >= need) return HE_OK;
    HE_TRY(he_capture_guard("polynomial temporaries"));
    for (he_ct *t : c->poly_tmp) he_ct_free(t);
    c->poly_tmp.clear();
    if (c->poly_block) he_free(c->poly_block);
    c->poly_block = nullptr;
    const size_t ps = (size_t)(c->L + 1) * c->n;
    HE_TRY(dev_alloc(&c->poly_block, need * 2 * ps));
    for (size_t i = 0; i < need; i++) {
        he_ct *t = nullptr;
        HE_TRY(he_ct_wrap(c, c->poly_block + i * 2 * ps, 2 * ps * 8, c->L, &t));
        c->poly_tmp.push_back(t);
    }
    return HE_OK;
}

// The Chebyshev tree on m ciphertexts at one level, side by side: every tree depth is one
// batched relinearisation over all of them (relin_batch), and each ciphertext gets exactly the
// bits the one-ciphertext evaluation gives it.  Temporaries poly_tmp[t0 .. t0 + m (2 deg + 4)).
static int poly_eval_group(he_ctx *c, const std::vector<he_ct *> &io, const double *cheb, int deg,
                           const std::vector<double> &tgt, size_t t0, cudaStream_t s) {
    const int m = (int)io.size();
    const size_t per = 2 * (size_t)deg + 4;
    int depth = 0;
    while ((1 << depth) < deg) depth++;
    std::vector<std::vector<he_ct *>> T(m), opA(m);
    std::vector<he_ct *> t1(m), acc(m), y(m);
    for (int j = 0; j < m; j++) {
        he_ct **tp = c->poly_tmp.data() + t0 + (size_t)j * per;
        T[j].assign(deg + 1, nullptr);
        opA[j].assign(deg + 1, nullptr);
        for (int k = 1; k <= deg; k++) T[j][k] = tp[k - 1];
        for (int k = 2; k <= deg; k++) opA[j][k] = tp[deg + k - 2];
        t1[j] = tp[2 * deg];
        acc[j] = tp[2 * deg + 1];
        y[j] = tp[2 * deg + 2];
        HE_TRY(he_ct_copy(T[j][1], io[j], s));
    }
    for (int d = 1; d <= depth; d++) {
        const int k0 = (1 << (d - 1)) + 1, k1 = std::min(deg, 1 << d);
        std::vector<const he_ct *> A, B;
        std::vector<he_ct *> O;
        for (int j = 0; j < m; j++)
            for (int k = k0; k <= k1; k++) {
                const int h = k / 2;
                if (k % 2 == 0) {
                    A.push_back(T[j][h]);
                    B.push_back(T[j][h]);
                } else {
                    // depth never decreases with k, so T_{h+1} already sits at the common level
                    // and only a copy of T_h is dropped to it
                    const int lv = T[j][h + 1]->level;
                    if (T[j][h]->level < lv) { he_set_error("he_poly_eval: operand levels out of order"); return HE_ESTATE; }
                    HE_TRY(he_ct_copy(opA[j][k], T[j][h], s));
                    HE_TRY(he_ct_drop_level(opA[j][k], lv));
                    A.push_back(opA[j][k]);
                    B.push_back(T[j][h + 1]);
                }
                O.push_back(T[j][k]);
            }
        HE_TRY(relin_batch(c, A, B, O, s));
        for (int j = 0; j < m; j++)
            for (int k = k0; k <= k1; k++) {
                HE_TRY(he_mul_int(c, T[j][k], 2.0, s));
                if (k % 2 == 0) {
                    HE_TRY(he_add_const_int(c, T[j][k], -std::nearbyint(T[j][k]->scale), s));
                } else {
                    HE_TRY(retarget(c, T[j][1], T[j][k]->level, T[j][k]->scale, t1[j], s));
                    HE_TRY(he_sub(c, T[j][k], t1[j], s));
                }
            }
    }
    for (int j = 0; j < m; j++) {
        const double target_scale = tgt[j];
        int lmin = T[j][1]->level;
        for (int k = 2; k <= deg; k++) lmin = std::min(lmin, T[j][k]->level);
        const double base = target_scale * (double)c->primes[lmin];
        const double cst = std::nearbyint(cheb[0] * target_scale * (double)c->primes[lmin]);
        if (deg <= 20 && lmin + 1 <= 24) {
            // one pass: acc = sum_k K_k T_k + c_0 (same integers and sums as the term-by-term form)
            std::vector<const u64 *> xs(deg);
            std::vector<size_t> pss(deg);
            std::vector<u64> res((size_t)deg * 24, 0), cres(24, 0);
            for (int k = 1; k <= deg; k++) {
                const double K = std::nearbyint(cheb[k] * target_scale * (double)c->primes[lmin] / T[j][k]->scale);
                xs[k - 1] = T[j][k]->d;
                pss[k - 1] = T[j][k]->pstride;
                for (int i = 0; i <= lmin; i++)
                    if (!int_residue(K, c->primes[i], &res[(size_t)(k - 1) * 24 + i])) {
                        he_set_error("he_poly_eval: constant is not an exact integer");
                        return HE_EINVAL;
                    }
            }
            for (int i = 0; i <= lmin; i++)
                if (!int_residue(cst, c->primes[i], &cres[i])) { he_set_error("he_poly_eval: bad constant"); return HE_EINVAL; }
            HE_TRY(ensure_ct(c, acc[j], lmin));
            HE_TRY(k_lincomb(c, xs.data(), pss.data(), res.data(), deg, cres.data(), lmin, acc[j]->d, acc[j]->pstride, s));
            acc[j]->scale = base;
            HE_TRY(he_rescale(c, acc[j], s));
            acc[j]->scale = target_scale;
            HE_TRY(he_ct_copy(io[j], acc[j], s));
            continue;
        }
        bool first = true;
        for (int k = 1; k <= deg; k++) {
            HE_TRY(he_ct_copy(y[j], T[j][k], s));
            HE_TRY(he_ct_drop_level(y[j], lmin));
            double K = std::nearbyint(cheb[k] * target_scale * (double)c->primes[lmin] / y[j]->scale);
            HE_TRY(he_mul_int(c, y[j], K, s));
            y[j]->scale = base;
            if (first) { HE_TRY(he_ct_copy(acc[j], y[j], s)); first = false; }
            else HE_TRY(he_add(c, acc[j], y[j], s));
        }
        HE_TRY(he_add_const_int(c, acc[j], cst, s));
        HE_TRY(he_rescale(c, acc[j], s));
        acc[j]->scale = target_scale;
        HE_TRY(he_ct_copy(io[j], acc[j], s));
    }
    return HE_OK;
}

// ---------------------------------------------------------------- Paterson-Stockmeyer
// sum c_j T_j in the Chebyshev basis with baby steps T_1..T_k and giant steps T_k, T_2k, ...
// (Appendix: the recursion T_{2n} = 2 T_n^2 - 1, T_{2n+1} = 2 T_n T_{n+1} - x builds both), and
// the division p = q T_G + r (T_G T_j = (T_{G+j} + T_{|G-j|}) / 2); every node is evaluated to a
// given (level, scale): leaves are exact-scale integer combinations, a product node lands its
// quotient one level up so that q T_G meets r on the same level and scale.  The operations and
// their order are the oracle's; every product is batched over the ciphertexts of a group.
static void ps_params(int deg, int &k, std::vector<int> &giants) {
    k = 2;
    while (k * k < (deg + 1) / 2) k *= 2;
    giants.clear();
    for (int g = k; g <= deg; g *= 2) giants.push_back(g);
}

static void cheb_divide(const std::vector<double> &c, int G, std::vector<double> &q, std::vector<double> &r) {
    const int d = (int)c.size() - 1;
    q.assign(1, c[G]);
    for (int j = 1; j <= d - G; j++) q.push_back(2.0 * c[G + j]);
    r.resize(G);
    for (int i = 0; i < G; i++) r[i] = c[i] - ((2 * G - i <= d && i >= 1) ? c[2 * G - i] : 0.0);
}

static int bit_len(int x) { int b = 0; while (x > 0) { b++; x >>= 1; } return b; }
static int ps_depth(int i) { return bit_len(i - 1); }         // level cost of T_i from the tree

static int ps_need(const std::vector<double> &cc, int k, const std::vector<int> &giants) {
    const int d = (int)cc.size() - 1;
    if (d < k) {
        int m = 0;
        for (int i = 1; i <= d; i++) m = std::max(m, ps_depth(i));
        return 1 + m;
    }
    int G = 0;
    for (int g : giants)
        if (g <= d) G = g;
    std::vector<double> q, r;
    cheb_divide(cc, G, q, r);
    if (q.size() == 1 && G - 1 < k) {
        int m = ps_depth(G);
        for (int i = 1; i < G; i++) m = std::max(m, ps_depth(i));
        return 1 + m;
    }
    if (q.size() == 1) return std::max(1 + ps_depth(G), ps_need(r, k, giants));
    return std::max(std::max(ps_need(q, k, giants) + 1, ps_depth(G) + 1), ps_need(r, k, giants));
}

// relinearised products of ev on a polynomial of degree d (the recursion of PsGroup::ev below):
// a split with a non-constant quotient costs its product plus the quotient's and remainder's
static int ps_split_products(int d, int k, const std::vector<int> &giants) {
    if (d < k) return 0;
    int G = 0;
    for (int g : giants)
        if (g <= d) G = g;
    if (d == G && G - 1 < k) return 0;                       // q_0 T_G + r in one combination
    if (d == G) return ps_split_products(G - 1, k, giants);  // scalar q_0 T_G plus ev(r)
    return 1 + ps_split_products(d - G, k, giants) + ps_split_products(G - 1, k, giants);
}

extern "C" int he_poly_ps_plan(int deg, int *products, int *depth) {
    if (deg < 2 || deg > 255) { he_set_error("he_poly_ps_plan: degree %d outside 2..255", deg); return HE_EINVAL; }
    int k;
    std::vector<int> giants;
    ps_params(deg, k, giants);
    int steps = 0;                                           // T_2..T_k and the giant steps beyond T_k
    const int top = std::max(k, giants.empty() ? 0 : giants.back());
    for (int i = 2; i <= top; i++)
        if (i <= k || std::find(giants.begin(), giants.end(), i) != giants.end()) steps++;
    if (products) *products = steps + ps_split_products(deg, k, giants);
    if (depth) *depth = ps_need(std::vector<double>(deg + 1, 1.0), k, giants);
    return HE_OK;
}

// sum_(coef, x) round(coef scale q_{l+1} / s_x) x + round(c0 scale q_{l+1}) at level l + 1, rescaled
// to (l, scale); y is scratch for the term-by-term form
// defer: stop before the rescale (out at level + 1, scale `scale` q_{l+1}); the caller rescales
// it, possibly together with other combinations of the same level, and sets the scale to `scale`
static int ps_lincomb(he_ctx *c, const std::vector<std::pair<double, const he_ct *>> &terms, double c0, int level,
                      double scale, he_ct *out, he_ct *y, cudaStream_t s, bool defer = false) {
    const int lm = level + 1;
    const double ql = (double)c->primes[lm];
    const double cst = std::nearbyint(c0 * scale * ql);
    if ((int)terms.size() <= HE_LC_MAX && lm + 1 <= HE_LC_LIMBS) {
        std::vector<const u64 *> xs;
        std::vector<size_t> pss;
        std::vector<u64> res((size_t)terms.size() * HE_LC_LIMBS, 0), cres(HE_LC_LIMBS, 0);
        for (size_t t = 0; t < terms.size(); t++) {
            const he_ct *x = terms[t].second;
            if (x->level < lm) { he_set_error("polynomial: operand below the combination level"); return HE_ESTATE; }
            const double K = std::nearbyint(terms[t].first * scale * ql / x->scale);
            xs.push_back(x->d);
            pss.push_back(x->pstride);
            for (int i = 0; i <= lm; i++)
                if (!int_residue(K, c->primes[i], &res[t * HE_LC_LIMBS + i])) {
                    he_set_error("polynomial: constant is not an exact integer");
                    return HE_EINVAL;
                }
        }
        for (int i = 0; i <= lm; i++)
            if (!int_residue(cst, c->primes[i], &cres[i])) { he_set_error("polynomial: bad constant"); return HE_EINVAL; }
        HE_TRY(ensure_ct(c, out, lm));
        HE_TRY(k_lincomb(c, xs.data(), pss.data(), res.data(), (int)terms.size(), cres.data(), lm, out->d,
                         out->pstride, s));
    } else {
        bool first = true;
        for (auto &tm : terms) {
            HE_TRY(he_ct_copy(y, tm.second, s));
            HE_TRY(he_ct_drop_level(y, lm));
            const double K = std::nearbyint(tm.first * scale * ql / y->scale);
            HE_TRY(he_mul_int(c, y, K, s));
            if (first) { HE_TRY(he_ct_copy(out, y, s)); first = false; }
            else HE_TRY(he_add(c, out, y, s));
        }
        HE_TRY(he_add_const_int(c, out, cst, s));
    }
    out->scale = scale * ql;
    if (defer) return HE_OK;
    HE_TRY(he_rescale(c, out, s));
    out->scale = scale;
    return HE_OK;
}

// Deferred Paterson-Stockmeyer evaluation.  The plan is recorded as operations, each with the
// ciphertexts it reads and writes; a scheduler then issues, pass after pass, every ready operation
// that is not a product (in program order), then every ready product of one level as one batched
// relinearisation.  An operation is ready when no earlier unfinished operation writes what it
// reads or touches what it writes, so every ciphertext gets the bits of the program-order
// evaluation; independent products of equal level (T_3 and T_4; the last giant step and the
// product inside a quotient; two sibling quotients' products) share one set of launches.
struct PsOp {
    bool prod = false;
    std::vector<const he_ct *> rd, wr;
    std::function<int()> fn;                                  // not a product
    std::function<void(he_ct &, he_ct &)> views;              // product operands, built at issue
    he_ct *out = nullptr;
    std::function<double()> expect;                           // product: predicted output scale
    bool done = false;
    // a combination whose final rescale the scheduler batches with the other ready combinations
    // of that level: fn leaves `rs` one level up and writes its target scale to *rs_scale
    he_ct *rs = nullptr;
    std::shared_ptr<double> rs_scale;
};

// A scale that is known once the ciphertexts in deps are computed.
struct PsScale {
    std::function<double()> f;
    std::vector<const he_ct *> deps;
};

static int ps_run(he_ctx *c, std::vector<PsOp> &ops, cudaStream_t s) {
    // dependencies from program order: an operation waits for the last writer of what it reads or
    // writes and, for what it writes, for the readers since that write.  Each of those waited in
    // turn for the writers and readers before it, so every earlier conflicting operation is done
    // once these are.
    std::vector<std::vector<size_t>> deps(ops.size());
    {
        std::map<const he_ct *, size_t> last_w;
        std::map<const he_ct *, std::vector<size_t>> readers;
        for (size_t i = 0; i < ops.size(); i++) {
            auto &d = deps[i];
            for (const he_ct *x : ops[i].rd) {
                auto w = last_w.find(x);
                if (w != last_w.end()) d.push_back(w->second);
            }
            for (const he_ct *x : ops[i].wr) {
                auto w = last_w.find(x);
                if (w != last_w.end()) d.push_back(w->second);
                auto r = readers.find(x);
                if (r != readers.end())
                    for (size_t j : r->second)
                        if (j != i) d.push_back(j);
            }
            for (const he_ct *x : ops[i].rd) readers[x].push_back(i);
            for (const he_ct *x : ops[i].wr) {
                last_w[x] = i;
                readers[x].clear();
            }
        }
    }
    auto ready = [&](size_t i) {
        for (size_t j : deps[i])
            if (!ops[j].done) return false;
        return true;
    };
    size_t left = ops.size();
    while (left) {
        bool moved = false;
        std::vector<size_t> rs_pend;                       // combinations awaiting their rescale
        for (size_t i = 0; i < ops.size(); i++)
            if (!ops[i].done && !ops[i].prod && ready(i)) {
                HE_TRY(ops[i].fn());
                if (ops[i].rs) {
                    rs_pend.push_back(i);
                    continue;
                }
                ops[i].done = true;
                left--;
                moved = true;
            }
        // one batched rescale per level for the combinations issued in this pass (ops that read
        // them were not ready, so nothing has used them yet)
        while (!rs_pend.empty()) {
            const int lv = ops[rs_pend[0]].rs->level;
            std::vector<size_t> here, rest;
            for (size_t i : rs_pend) (ops[i].rs->level == lv ? here : rest).push_back(i);
            std::vector<he_ct *> grp;
            for (size_t i : here) grp.push_back(ops[i].rs);
            HE_TRY(rescale_batch(c, grp.data(), (int)grp.size(), s));
            for (size_t i : here) {
                ops[i].rs->scale = *ops[i].rs_scale;
                ops[i].done = true;
                left--;
            }
            moved = true;
            rs_pend = rest;
        }
        std::vector<size_t> P;
        std::vector<he_ct> va, vb;
        int lv = -1;
        for (size_t i = 0; i < ops.size(); i++) {
            if (ops[i].done || !ops[i].prod || !ready(i)) continue;
            he_ct a, b;
            ops[i].views(a, b);
            if (a.level != b.level) { he_set_error("polynomial: product operands at levels %d and %d", a.level, b.level); return HE_ESTATE; }
            if (lv < 0) lv = a.level;
            if (a.level != lv) continue;
            P.push_back(i);
            va.push_back(a);
            vb.push_back(b);
        }
        if (!P.empty()) {
            std::vector<const he_ct *> A, B;
            std::vector<he_ct *> O;
            for (size_t k = 0; k < P.size(); k++) {
                A.push_back(&va[k]);
                B.push_back(&vb[k]);
                O.push_back(ops[P[k]].out);
            }
            HE_TRY(relin_batch(c, A, B, O, s));
            for (size_t k = 0; k < P.size(); k++) {
                PsOp &o = ops[P[k]];
                if (o.expect && o.out->scale != o.expect()) { he_set_error("polynomial: product scale off its prediction"); return HE_ESTATE; }
                o.done = true;
                left--;
            }
            moved = true;
        }
        if (!moved) { he_set_error("polynomial: schedule stalled"); return HE_ESTATE; }
    }
    return HE_OK;
}

struct PsGroup {
    he_ctx *c;
    cudaStream_t s;
    int k;
    std::vector<int> giants;
    int m;
    std::vector<std::map<int, he_ct *>> T;                   // per ciphertext: index -> T_index
    std::vector<std::vector<he_ct *>> tq, tr;                // per ciphertext, per recursion depth
    std::vector<he_ct *> t1, y;
    std::vector<PsOp> ops;

    // a linear combination of T's (scratch y only where ps_lincomb takes its term-by-term form)
    void lincomb(int j, std::vector<std::pair<double, int>> terms, double c0, int level, const PsScale &sc,
                 he_ct *out) {
        PsOp o;
        for (auto &t : terms) o.rd.push_back(T[j][t.second]);
        for (auto *d : sc.deps) o.rd.push_back(d);
        o.wr.push_back(out);
        if (!((int)terms.size() <= HE_LC_MAX && level + 2 <= HE_LC_LIMBS)) o.wr.push_back(y[j]);
        he_ctx *cc = c;
        cudaStream_t st = s;
        std::vector<std::pair<double, const he_ct *>> tv;
        for (auto &t : terms) tv.push_back({t.first, T[j][t.second]});
        he_ct *yj = y[j];
        std::function<double()> f = sc.f;
        auto rs_scale = std::make_shared<double>(0.0);
        o.rs = out;
        o.rs_scale = rs_scale;
        o.fn = [cc, st, tv, c0, level, f, out, yj, rs_scale]() {
            *rs_scale = f();
            return ps_lincomb(cc, tv, c0, level, *rs_scale, out, yj, st, true);
        };
        ops.push_back(std::move(o));
    }
    void add(he_ct *acc, he_ct *b) {
        PsOp o;
        o.rd = {acc, b};
        o.wr = {acc};
        he_ctx *cc = c;
        cudaStream_t st = s;
        o.fn = [cc, st, acc, b]() { return he_add(cc, acc, b, st); };
        ops.push_back(std::move(o));
    }

    // records the evaluation of sum cc_i T_i into out at (level, sc); returns the result's scale
    std::vector<PsScale> ev(const std::vector<double> &cc, int level, const std::vector<PsScale> &sc,
                            const std::vector<he_ct *> &out, int depth) {
        const int d = (int)cc.size() - 1;
        if (d < k) {
            for (int j = 0; j < m; j++) {
                std::vector<std::pair<double, int>> terms;
                for (int i = 1; i <= d; i++) terms.push_back({cc[i], i});
                lincomb(j, terms, cc[0], level, sc[j], out[j]);
            }
            return sc;
        }
        int G = 0;
        for (int g : giants)
            if (g <= d) G = g;
        std::vector<double> q, r;
        cheb_divide(cc, G, q, r);
        if (q.size() == 1 && G - 1 < k) {                    // q_0 T_G + r in one combination
            for (int j = 0; j < m; j++) {
                std::vector<std::pair<double, int>> terms;
                for (int i = 1; i < G; i++) terms.push_back({r[i], i});
                terms.push_back({q[0], G});
                lincomb(j, terms, r[0], level, sc[j], out[j]);
            }
            return sc;
        }
        if (q.size() == 1) {                                 // ev(r) plus the scalar q_0 T_G
            std::vector<PsScale> res = ev(r, level, sc, out, depth + 1);
            for (int j = 0; j < m; j++) {
                lincomb(j, {{q[0], G}}, 0.0, level, sc[j], tq[j][depth]);
                add(out[j], tq[j][depth]);
            }
            return res;
        }
        // q T_G + r: the quotient one level up, its product with T_G (dropped to level + 1), then
        // the remainder at the product's scale
        const double ql1 = (double)c->primes[level + 1];
        std::vector<PsScale> sq(m);
        std::vector<he_ct *> qo(m), ro(m);
        for (int j = 0; j < m; j++) {
            const he_ct *TG = T[j][G];
            std::function<double()> f = sc[j].f;
            sq[j].f = [f, ql1, TG]() { return f() * ql1 / TG->scale; };
            sq[j].deps = sc[j].deps;
            sq[j].deps.push_back(TG);
            qo[j] = tq[j][depth];
            ro[j] = tr[j][depth];
        }
        std::vector<PsScale> resq = ev(q, level + 1, sq, qo, depth + 1);
        std::vector<PsScale> ps_(m);
        for (int j = 0; j < m; j++) {
            const he_ct *TG = T[j][G];
            he_ct *a = qo[j];
            const int lp1 = level + 1;
            PsOp o;
            o.prod = true;
            o.rd = {a, TG};
            o.wr = {out[j]};
            o.out = out[j];
            o.views = [a, TG, lp1](he_ct &A, he_ct &B) {
                A = *a;
                B = *TG;                                     // T_G dropped to level + 1 (a view)
                B.level = lp1;
            };
            std::function<double()> fq = resq[j].f;
            // relin_batch's own arithmetic: (s_A s_B) / q_{level+1}
            o.expect = [fq, TG, ql1]() {
                double t = fq() * TG->scale;
                return t / ql1;
            };
            ps_[j].f = o.expect;
            ps_[j].deps = resq[j].deps;
            ps_[j].deps.push_back(TG);
            ops.push_back(std::move(o));
        }
        ev(r, level, ps_, ro, depth + 1);
        for (int j = 0; j < m; j++) add(out[j], ro[j]);
        return ps_;
    }
};

// m ciphertexts at one level; temporaries poly_tmp[t0 .. t0 + m * per)
static int ps_group(he_ctx *c, const std::vector<he_ct *> &io, const double *cheb, int deg,
                    const std::vector<double> &tgt, size_t t0, size_t per, cudaStream_t s) {
    PsGroup P;
    P.c = c;
    P.s = s;
    P.m = (int)io.size();
    ps_params(deg, P.k, P.giants);
    std::vector<double> cc(cheb, cheb + deg + 1);
    const int need = ps_need(cc, P.k, P.giants);
    const int lin = io[0]->level;
    if (lin - need < 0) { he_set_error("he_poly_eval_ps: needs %d levels", need); return HE_ELEVEL; }
    std::vector<int> idx;
    const int top = std::max(P.k, P.giants.empty() ? 0 : P.giants.back());
    for (int i = 1; i <= top; i++)
        if (i <= P.k || std::find(P.giants.begin(), P.giants.end(), i) != P.giants.end()) idx.push_back(i);
    const int nd = (int)P.giants.size() + 2;
    P.T.resize(P.m);
    P.tq.resize(P.m);
    P.tr.resize(P.m);
    P.t1.resize(P.m);
    P.y.resize(P.m);
    std::vector<he_ct *> outv(P.m);
    for (int j = 0; j < P.m; j++) {
        he_ct **tp = c->poly_tmp.data() + t0 + (size_t)j * per;
        size_t u = 0;
        for (int i : idx) P.T[j][i] = tp[u++];
        for (int d = 0; d < nd; d++) {
            P.tq[j].push_back(tp[u++]);
            P.tr[j].push_back(tp[u++]);
        }
        P.t1[j] = tp[u++];
        P.y[j] = tp[u++];
        outv[j] = tp[u++];
        if (u > per) { he_set_error("polynomial: temporaries"); return HE_ESTATE; }
        HE_TRY(he_ct_copy(P.T[j][1], io[j], s));
    }
    // baby and giant steps: T_2h = 2 T_h^2 - 1, T_2h+1 = 2 T_h T_h+1 - T_1 (operands dropped to the
    // lower of their levels)
    for (int i : idx) {
        if (i == 1) continue;
        const int h = i / 2;
        for (int j = 0; j < P.m; j++) {
            he_ct *Th = P.T[j][h], *Ti = P.T[j][i], *T1 = P.T[j][1], *t1 = P.t1[j];
            he_ct *Th1 = i % 2 ? P.T[j][h + 1] : nullptr;
            PsOp o;
            o.prod = true;
            o.out = Ti;
            o.wr = {Ti};
            if (i % 2 == 0) {
                o.rd = {Th};
                o.views = [Th](he_ct &A, he_ct &B) { A = *Th; B = *Th; };
            } else {
                o.rd = {Th, Th1};
                o.views = [Th, Th1](he_ct &A, he_ct &B) {
                    const int lv = std::min(Th->level, Th1->level);
                    A = *Th;
                    A.level = lv;
                    B = *Th1;
                    B.level = lv;
                };
            }
            P.ops.push_back(std::move(o));
            PsOp f;
            f.rd = {Ti, T1};
            f.wr = {Ti};
            if (i % 2) f.wr.push_back(t1);
            const bool even = i % 2 == 0;
            f.fn = [c, s, Ti, T1, t1, even]() {
                HE_TRY(he_mul_int(c, Ti, 2.0, s));
                if (even) return he_add_const_int(c, Ti, -std::nearbyint(Ti->scale), s);
                HE_TRY(retarget(c, T1, Ti->level, Ti->scale, t1, s));
                return he_sub(c, Ti, t1, s);
            };
            P.ops.push_back(std::move(f));
        }
    }
    std::vector<PsScale> sc(P.m);
    for (int j = 0; j < P.m; j++) {
        const double v = tgt[j];
        sc[j].f = [v]() { return v; };
    }
    P.ev(cc, lin - need, sc, outv, 0);
    HE_TRY(ps_run(c, P.ops, s));
    for (int j = 0; j < P.m; j++) HE_TRY(he_ct_copy(io[j], outv[j], s));
    return HE_OK;
}

extern "C" int he_poly_eval_ps_many(he_ctx *c, he_ct *const *io, int m, const double *cheb, int deg,
                                    const double *target_scales, void *stream) {
    if (!c || !io || m < 1 || !cheb || !target_scales || deg < 2 || deg > 255) {
        he_set_error("he_poly_eval_ps_many: bad argument");
        return HE_EINVAL;
    }
    int k;
    std::vector<int> giants;
    ps_params(deg, k, giants);
    const size_t per = (size_t)k + giants.size() + 2 * (giants.size() + 2) + 3;
    std::map<int, std::vector<int>> by_level;
    for (int j = 0; j < m; j++) {
        if (!io[j] || io[j]->ctx != c) { he_set_error("he_poly_eval_ps_many: ciphertext %d missing", j); return HE_EINVAL; }
        by_level[io[j]->level].push_back(j);
    }
    HE_TRY(poly_temps(c, (size_t)m * per));
    size_t t0 = 0;
    for (auto &kv : by_level) {
        std::vector<he_ct *> grp;
        std::vector<double> tg;
        for (int j : kv.second) {
            grp.push_back(io[j]);
            tg.push_back(target_scales[j]);
        }
        HE_TRY(ps_group(c, grp, cheb, deg, tg, t0, per, (cudaStream_t)stream));
        t0 += grp.size() * per;
    }
    return HE_OK;
}

extern "C" int he_poly_eval_ps(he_ctx *c, he_ct *io, const double *cheb, int deg, double target_scale, void *stream) {
    he_ct *a[1] = {io};
    return he_poly_eval_ps_many(c, a, 1, cheb, deg, &target_scale, stream);
}

extern "C" int he_poly_eval(he_ctx *c, he_ct *io, const double *cheb, int deg, double target_scale, void *stream) {
    if (!c || !io || !cheb || deg < 1 || deg > 64) { he_set_error("he_poly_eval: bad argument"); return HE_EINVAL; }
    int depth = 0;
    while ((1 << depth) < deg) depth++;
    if (io->level < depth + 1) { he_set_error("he_poly_eval: needs %d levels", depth + 1); return HE_ELEVEL; }
    HE_TRY(poly_temps(c, 2 * (size_t)deg + 4));
    return poly_eval_group(c, {io}, cheb, deg, {target_scale}, 0, (cudaStream_t)stream);
}

extern "C" int he_poly_eval_many(he_ctx *c, he_ct *const *io, int m, const double *cheb, int deg,
                                 const double *target_scales, void *stream) {
    if (!c || !io || m < 1 || !cheb || !target_scales || deg < 1 || deg > 64) {
        he_set_error("he_poly_eval_many: bad argument");
        return HE_EINVAL;
    }
    int depth = 0;
    while ((1 << depth) < deg) depth++;
    std::map<int, std::vector<int>> by_level;
    for (int j = 0; j < m; j++) {
        if (!io[j] || io[j]->ctx != c) { he_set_error("he_poly_eval_many: ciphertext %d missing", j); return HE_EINVAL; }
        if (io[j]->level < depth + 1) { he_set_error("he_poly_eval: needs %d levels", depth + 1); return HE_ELEVEL; }
        by_level[io[j]->level].push_back(j);
    }
    const size_t per = 2 * (size_t)deg + 4;
    HE_TRY(poly_temps(c, (size_t)m * per));
    size_t t0 = 0;
    for (auto &kv : by_level) {
        std::vector<he_ct *> grp;
        std::vector<double> tg;
        for (int j : kv.second) {
            grp.push_back(io[j]);
            tg.push_back(target_scales[j]);
        }
        HE_TRY(poly_eval_group(c, grp, cheb, deg, tg, t0, (cudaStream_t)stream));
        t0 += grp.size() * per;
    }
    return HE_OK;
}

// ================================================================================ linear head
// Linear layer over a sharded image (Sec. 4 "Other Layers", Linear): T_j = Rescale(sum_u w_{j,u}
// (.) X_u) with row j of the weights on the first copy of every valid pixel (scale q_l); for
// s = N/2, ..., 1: T_j += rot_s(T_j) (one fused raised-basis stage per shift over every j: the
// shift key is read once for all outputs, and each output takes one ModDown, which gives the
// bits of T_j + hoisted rotation); out = Rescale(sum_j e_j (.) T_j) with the one-hot masks at
// scale q_{l-1}, plus the bias in slots 0..n_out-1.  Pool-linear spreads per-channel weights over
// the m x m pixels, divided by m^2.
// The slot sum adds every slot of a partial sum, each of its steps doubling the noise of the key
// switches before it, so it runs at scale Delta 2^12: weights at q_l 2^12, masks at
// q_{l-1} / 2^12 (the output is back at Delta exactly).
constexpr int HEAD_BOOST_BITS = 12;
static double head_w_scale(const he_ctx *c, int l) { return (double)c->primes[l] * std::ldexp(1.0, HEAD_BOOST_BITS); }
static double head_mask_scale(const he_ctx *c, int l) { return (double)c->primes[l - 1] / std::ldexp(1.0, HEAD_BOOST_BITS); }

struct he_linear {
    he_ctx *c = nullptr;
    Lay lin;
    int n_out = 0, level = 0;
    double in_scale = 1.0;
    size_t pw = 0;                               // poly stride of every buffer: level l
    std::vector<double> bias;
    u64 *R = nullptr;                            // [n_in][2][pw] input copies
    u64 *w = nullptr;                            // [n_out][n_in][pw] weights, Montgomery NTT form
    u64 *mask = nullptr;                         // [n_out][l][n] masks at level l - 1
    u64 *bias_pt = nullptr;                      // [l - 1][n] bias addend at level l - 2
    u64 *T[2] = {nullptr, nullptr};              // [n_out][2][pw] partial sums (ping-pong)
    u64 *acc = nullptr;                          // [2][pw]
    mac_term *d_w = nullptr, *d_m = nullptr;     // weight MACs; mask MACs (over the final T)
    std::vector<std::unique_ptr<FusedStage>> steps;
    std::vector<int> shifts;
    // packed form: one sum C = sum_{(u,d)} Q_{u,d} (.) rot_d(X_u) (a raised-basis stage, d < npk)
    // whose slot classes mod npk are summed by the shifts N/2, ..., npk; w holds the Q_{u,d}
    // ([n_in][npk][l+1+K][n]), mask the single first-n_out mask, T one partial sum
    bool packed = false;
    int npk = 0;
    std::unique_ptr<FusedStage> stage1;
    int n_T() const { return packed ? 1 : n_out; }    // partial sums held
    ~he_linear() {
        cudaDeviceSynchronize();
        steps.clear();
        stage1.reset();
        he_free(R); he_free(w); he_free(mask); he_free(bias_pt); he_free(T[0]); he_free(T[1]);
        he_free(acc); he_free(d_w); he_free(d_m);
    }
};

// row j of the weights on the first copy of every valid pixel of shard u; W[j][c][m][m]
static void linear_weights(const Lay &L, const double *W, int j, int u, const std::vector<char> &first,
                           std::vector<double> &out) {
    out.assign(L.N, 0.0);
    for (int i = 0; i < L.N; i++) {
        if (!first[(size_t)u * L.N + i]) continue;
        SlotInfo si = slot_info(L, u, i);
        out[i] = W[(((size_t)j * L.c + si.ch) * L.m + si.y) * L.m + si.x];
    }
}

static int linear_create(he_ctx *c, const he_layout *in, const double *W, const double *bias, int n_out, int level,
                         double in_scale, bool packed, he_linear **out) {
    if (!c || !in || !W || !out || n_out < 1) { he_set_error("he_linear_create: bad argument"); return HE_EINVAL; }
    if (level < 2 || level > c->L) { he_set_error("he_linear_create: level %d, the head takes two levels", level); return HE_ELEVEL; }
    Lay lin = from_c(*in);
    HE_TRY(check_layout(lin, c->N));
    if (n_out > lin.N) { he_set_error("he_linear_create: %d outputs exceed %d slots", n_out, lin.N); return HE_EINVAL; }
    std::unique_ptr<he_linear> L(new he_linear());
    L->c = c;
    L->lin = lin;
    L->n_out = n_out;
    L->level = level;
    L->in_scale = in_scale;
    L->pw = (size_t)(level + 1) * c->n;
    L->bias.assign(n_out, 0.0);
    if (bias) L->bias.assign(bias, bias + n_out);
    L->packed = packed;
    L->npk = 1;
    while (L->npk < n_out) L->npk *= 2;
    for (int s = lin.N / 2; s >= (packed ? L->npk : 1); s /= 2) L->shifts.push_back(s);
    const int ni = lin.ns, n = c->n;
    // first copy (shard, then block order) of every (channel, row, column)
    std::vector<char> first((size_t)ni * lin.N, 0), seen((size_t)lin.c * lin.m * lin.m, 0);
    for (int u = 0; u < ni; u++)
        for (int i = 0; i < lin.N; i++) {
            SlotInfo si = slot_info(lin, u, i);
            if (!si.valid) continue;
            char &sn = seen[((size_t)si.ch * lin.m + si.y) * lin.m + si.x];
            if (!sn) { sn = 1; first[(size_t)u * lin.N + i] = 1; }
        }
    HE_TRY(dev_alloc(&L->R, (size_t)ni * 2 * L->pw));
    HE_TRY(dev_alloc(&L->bias_pt, (size_t)(level - 1) * n));
    for (int b = 0; b < 2; b++) HE_TRY(dev_alloc(&L->T[b], (size_t)L->n_T() * 2 * L->pw));
    HE_TRY(dev_alloc(&L->acc, 2 * L->pw));
    {
        std::vector<double> z(lin.N, 0.0);
        for (int j = 0; j < n_out; j++) z[j] = L->bias[j];
        std::vector<int64_t> m(n);
        encode_slots(z.data(), n, in_scale, m.data());
        HE_TRY(upload_addend(c, m.data(), level - 2, L->bias_pt));
    }
    if (packed) {
        // Q_{u,d}[i] = w_{i mod npk, u}[(i + d) mod N] (zero rows past n_out), raised layout
        const int np = L->npk, N = lin.N;
        const size_t pe = (size_t)(level + 1 + c->K) * n;
        HE_TRY(dev_alloc(&L->w, (size_t)ni * np * pe));
        HE_TRY(dev_alloc(&L->mask, (size_t)level * n));
        std::vector<std::vector<double>> rows(n_out);
        std::vector<std::vector<double>> Q(np, std::vector<double>(N));
        for (int u = 0; u < ni; u++) {
            for (int j = 0; j < n_out; j++) linear_weights(lin, W, j, u, first, rows[j]);
            std::vector<const double *> vecs;
            for (int d = 0; d < np; d++) {
                for (int i = 0; i < N; i++) {
                    const int j = i % np;
                    Q[d][i] = j < n_out ? rows[j][(i + d) % N] : 0.0;
                }
                vecs.push_back(Q[d].data());
            }
            HE_TRY(upload_plaintexts(c, vecs, np, head_w_scale(c, level), level, L->w + (size_t)u * np * pe, nullptr,
                                     true));
        }
        std::vector<double> e(N, 0.0);
        for (int j = 0; j < n_out; j++) e[j] = 1.0;
        std::vector<const double *> vecs{e.data()};
        HE_TRY(upload_plaintexts(c, vecs, 1, head_mask_scale(c, level), level - 1, L->mask, nullptr));
        mac_term tm{L->mask, L->T[L->shifts.size() % 2], L->pw};
        HE_TRY(dev_alloc(&L->d_m, 1));
        HE_CHECK_CUDA(cudaMemcpy(L->d_m, &tm, sizeof(mac_term), cudaMemcpyHostToDevice));
        *out = L.release();
        return HE_OK;
    }
    HE_TRY(dev_alloc(&L->w, (size_t)n_out * ni * L->pw));
    HE_TRY(dev_alloc(&L->mask, (size_t)n_out * level * n));
    std::vector<std::vector<double>> rows(ni);
    for (int j = 0; j < n_out; j++) {
        std::vector<const double *> vecs;
        for (int u = 0; u < ni; u++) {
            linear_weights(lin, W, j, u, first, rows[u]);
            vecs.push_back(rows[u].data());
        }
        HE_TRY(upload_plaintexts(c, vecs, ni, head_w_scale(c, level), level, L->w + (size_t)j * ni * L->pw, nullptr));
    }
    std::vector<double> e(lin.N, 0.0);
    for (int j = 0; j < n_out; j++) {
        e.assign(lin.N, 0.0);
        e[j] = 1.0;
        std::vector<const double *> vecs{e.data()};
        HE_TRY(upload_plaintexts(c, vecs, 1, head_mask_scale(c, level), level - 1, L->mask + (size_t)j * level * n,
                                 nullptr));
    }
    // MAC tables: weights over the input copies; masks over the partial sums after the last shift
    std::vector<mac_term> tw((size_t)n_out * ni), tm(n_out);
    for (int j = 0; j < n_out; j++)
        for (int u = 0; u < ni; u++)
            tw[(size_t)j * ni + u] = mac_term{L->w + ((size_t)j * ni + u) * L->pw, L->R + (size_t)u * 2 * L->pw, L->pw};
    const int fin = (int)(L->shifts.size() % 2);      // buffer holding T after the last shift
    for (int j = 0; j < n_out; j++)
        tm[j] = mac_term{L->mask + (size_t)j * level * n, L->T[fin] + (size_t)j * 2 * L->pw, L->pw};
    HE_TRY(dev_alloc(&L->d_w, tw.size()));
    HE_TRY(dev_alloc(&L->d_m, tm.size()));
    HE_CHECK_CUDA(cudaMemcpy(L->d_w, tw.data(), tw.size() * sizeof(mac_term), cudaMemcpyHostToDevice));
    HE_CHECK_CUDA(cudaMemcpy(L->d_m, tm.data(), tm.size() * sizeof(mac_term), cudaMemcpyHostToDevice));
    *out = L.release();
    return HE_OK;
}

extern "C" int he_linear_create(he_ctx *c, const he_layout *in, const double *W, const double *bias, int n_out,
                                int level, double in_scale, he_linear **out) {
    return linear_create(c, in, W, bias, n_out, level, in_scale, false, out);
}

extern "C" int he_linear_create_packed(he_ctx *c, const he_layout *in, const double *W, const double *bias, int n_out,
                                       int level, double in_scale, he_linear **out) {
    return linear_create(c, in, W, bias, n_out, level, in_scale, true, out);
}

static int pool_linear_create(he_ctx *c, const he_layout *in, const double *W, const double *bias, int n_out,
                              int level, double in_scale, bool packed, he_linear **out);

extern "C" int he_pool_linear_create(he_ctx *c, const he_layout *in, const double *W, const double *bias, int n_out,
                                     int level, double in_scale, he_linear **out) {
    return pool_linear_create(c, in, W, bias, n_out, level, in_scale, false, out);
}

extern "C" int he_pool_linear_create_packed(he_ctx *c, const he_layout *in, const double *W, const double *bias,
                                            int n_out, int level, double in_scale, he_linear **out) {
    return pool_linear_create(c, in, W, bias, n_out, level, in_scale, true, out);
}

static int pool_linear_create(he_ctx *c, const he_layout *in, const double *W, const double *bias, int n_out,
                              int level, double in_scale, bool packed, he_linear **out) {
    if (!in || !W || n_out < 1 || in->c < 1 || in->m < 1) { he_set_error("he_pool_linear_create: bad argument"); return HE_EINVAL; }
    const int C = in->c, m = in->m;
    std::vector<double> full((size_t)n_out * C * m * m);
    const double norm = 1.0 / ((double)m * m);
    for (int j = 0; j < n_out; j++)
        for (int f = 0; f < C; f++)
            for (int k = 0; k < m * m; k++) full[((size_t)j * C + f) * m * m + k] = W[(size_t)j * C + f] * norm;
    return linear_create(c, in, full.data(), bias, n_out, level, in_scale, packed, out);
}

extern "C" void he_linear_destroy(he_linear *L) { delete L; }

extern "C" int he_linear_rotations(const he_linear *L, int32_t *amounts, size_t cap) {
    if (!L) return HE_EINVAL;
    std::vector<int> v;
    if (L->packed)
        for (int d = 1; d < L->npk; d++) v.push_back(d);
    v.insert(v.end(), L->shifts.begin(), L->shifts.end());
    for (size_t i = 0; i < v.size() && i < cap; i++) amounts[i] = v[i];
    return (int)v.size();
}

extern "C" int he_linear_out_level(const he_linear *L) { return L ? L->level - 2 : HE_EINVAL; }

extern "C" int64_t he_linear_keyswitches(const he_linear *L) {
    if (!L) return HE_EINVAL;
    if (L->packed) return (int64_t)L->lin.ns * (L->npk - 1) + (int64_t)L->shifts.size();
    return (int64_t)L->n_out * (int64_t)L->shifts.size();
}

extern "C" int he_linear_import_plaintexts(he_linear *L, const int64_t *weights, const int64_t *masks,
                                           const int64_t *bias) {
    if (!L) return HE_EINVAL;
    he_ctx *c = L->c;
    const int ni = L->lin.ns, n = c->n;
    std::vector<const double *> none;
    if (L->packed) {                              // weights [n_in][npk][n], mask [1][n]
        const size_t pe = (size_t)(L->level + 1 + c->K) * n;
        if (weights)
            for (int u = 0; u < ni; u++)
                HE_TRY(upload_plaintexts(c, none, L->npk, 0.0, L->level, L->w + (size_t)u * L->npk * pe,
                                         weights + (size_t)u * L->npk * n, true));
        if (masks) HE_TRY(upload_plaintexts(c, none, 1, 0.0, L->level - 1, L->mask, masks));
        if (bias) HE_TRY(upload_addend(c, bias, L->level - 2, L->bias_pt));
        if (weights && L->stage1) L->stage1->invalidate_pk();
        return HE_OK;
    }
    if (weights)
        for (int j = 0; j < L->n_out; j++)
            HE_TRY(upload_plaintexts(c, none, ni, 0.0, L->level, L->w + (size_t)j * ni * L->pw,
                                     weights + (size_t)j * ni * n));
    if (masks)
        for (int j = 0; j < L->n_out; j++)
            HE_TRY(upload_plaintexts(c, none, 1, 0.0, L->level - 1, L->mask + (size_t)j * L->level * n,
                                     masks + (size_t)j * n));
    if (bias) HE_TRY(upload_addend(c, bias, L->level - 2, L->bias_pt));
    return HE_OK;
}

// one fused stage per shift: sources T[b], outputs T[1-b], terms (j, j, 0, 1) and (j, j, s, 1)
static int linear_steps(he_linear *L) {
    if (!L->steps.empty()) return HE_OK;
    HE_TRY(he_capture_guard("the linear head's first run"));
    for (size_t k = 0; k < L->shifts.size(); k++) {
        std::unique_ptr<FusedStage> F(new FusedStage());
        F->c = L->c;
        F->level = L->level - 1;
        F->name = "linear head shift " + std::to_string(L->shifts[k]);
        u64 *src = L->T[k % 2], *dst = L->T[(k + 1) % 2];
        for (int j = 0; j < L->n_T(); j++) {
            F->add_src(src + (size_t)j * 2 * L->pw, L->pw);
            F->add_out(dst + (size_t)j * 2 * L->pw, L->pw);
        }
        for (int j = 0; j < L->n_T(); j++) {
            F->add_term(j, j, 0, HE_PT_ONE);
            F->add_term(j, j, L->shifts[k], HE_PT_ONE);
        }
        HE_TRY(F->build());
        L->steps.push_back(std::move(F));
    }
    if (L->packed) {                              // C = sum_{(u,d)} Q_{u,d} (.) rot_d(X_u), raised
        std::unique_ptr<FusedStage> F(new FusedStage());
        F->c = L->c;
        F->level = L->level;
        F->name = "packed linear head";
        const size_t pe = (size_t)(L->level + 1 + L->c->K) * L->c->n;
        for (int u = 0; u < L->lin.ns; u++) F->add_src(L->R + (size_t)u * 2 * L->pw, L->pw);
        F->add_out(L->T[0], L->pw);
        for (int u = 0; u < L->lin.ns; u++)
            for (int d = 0; d < L->npk; d++) F->add_term(0, u, d, L->w + ((size_t)u * L->npk + d) * pe);
        HE_TRY(F->build());
        L->stage1 = std::move(F);
    }
    return HE_OK;
}

extern "C" int he_linear_run(he_ctx *c, he_linear *L, he_ct *const *in, he_ct *out, void *stream) {
    if (!c || !L || !in || !out || L->c != c || out->ctx != c) { he_set_error("he_linear_run: bad argument"); return HE_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const int lv = L->level, ni = L->lin.ns;
    const size_t pw = L->pw;
    for (int u = 0; u < ni; u++) {
        if (!in[u] || in[u]->ctx != c || in[u]->level != lv || in[u]->scale != L->in_scale) {
            he_set_error("he_linear_run: input shard %d is not at level %d / the planned scale", u, lv);
            return HE_ELEVEL;
        }
        HE_TRY(k_copy_limbs(L->R + (size_t)u * 2 * pw, pw, in[u]->d, in[u]->pstride, pw, 2, s));
    }
    HE_TRY(linear_steps(L));
    if (L->packed) {                              // C, rescaled
        HE_TRY(L->stage1->run(s));
        he_ct v = view(c, L->T[0], pw, lv, L->in_scale * head_w_scale(c, lv));
        HE_TRY(he_rescale(c, &v, stream));
    }
    // T_j = Rescale(sum_u w_{j,u} (.) X_u)
    for (int j = 0; j < (L->packed ? 0 : L->n_out); j++) {
        u64 *t = L->T[0] + (size_t)j * 2 * pw;
        HE_TRY(k_mac(c, L->d_w + (size_t)j * ni, ni, t, pw, lv, false, s));
        he_ct v = view(c, t, pw, lv, L->in_scale * head_w_scale(c, lv));
        HE_TRY(he_rescale(c, &v, stream));
    }
    for (auto &F : L->steps) HE_TRY(F->run(s));
    // out = Rescale(sum_j e_j (.) T_j) + bias
    HE_TRY(k_mac(c, L->d_m, L->n_T(), L->acc, pw, lv - 1, false, s));
    const double t_scale = L->in_scale * head_w_scale(c, lv) / (double)c->primes[lv];
    he_ct v = view(c, L->acc, pw, lv - 1, t_scale * head_mask_scale(c, lv));
    HE_TRY(he_rescale(c, &v, stream));
    HE_TRY(k_add_raw(c, L->acc, pw, L->bias_pt, 0, lv - 1, 1, false, s));
    HE_TRY(ensure_ct(c, out, lv - 2));
    HE_TRY(k_copy_limbs(out->d, out->pstride, L->acc, pw, (size_t)(lv - 1) * c->n, 2, s));
    out->scale = v.scale;
    return HE_OK;
}

// ================================================================================ wrappers
static int keygen_for(he_ctx *c, const std::vector<int32_t> &amts) {
    return he_keygen_rotations(c, amts.data(), amts.size());
}

extern "C" int he_hconv2d(he_ctx *c, const he_layout *in, he_ct *const *in_cts, const double *W,
                          const double *bias, int co, int ci, int kh, int kw, int stride, int pad,
                          int mode, he_layout *out_layout, he_ct **out_cts, void *stream) {
    if (!c || !in || !in_cts || !out_cts) { he_set_error("null argument"); return HE_EINVAL; }
    he_conv *cv = nullptr;
    HE_TRY(he_conv_create(c, in, W, bias, co, ci, kh, kw, stride, pad, in_cts[0]->level, in_cts[0]->scale, &cv));
    int n = he_conv_rotations(cv, nullptr, 0);
    std::vector<int32_t> amts(std::max(n, 0));
    he_conv_rotations(cv, amts.data(), amts.size());
    int rc = keygen_for(c, amts);
    if (rc == HE_OK && out_layout) rc = he_conv_out_layout(cv, out_layout);
    if (rc == HE_OK) rc = he_conv_run(c, cv, in_cts, out_cts, mode, stream);
    if (rc == HE_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) rc = HE_ECUDA;
    he_conv_destroy(cv);
    return rc;
}

extern "C" int he_havgpool(he_ctx *c, const he_layout *in, he_ct *const *in_cts, he_layout *out_layout,
                           he_ct **out_cts, int mode, void *stream) {
    if (!c || !in || !in_cts || !out_cts) { he_set_error("null argument"); return HE_EINVAL; }
    he_pool *p = nullptr;
    HE_TRY(he_pool_create(c, in, in_cts[0]->level, &p));
    int n = he_pool_rotations(p, nullptr, 0);
    std::vector<int32_t> amts(std::max(n, 0));
    he_pool_rotations(p, amts.data(), amts.size());
    int rc = keygen_for(c, amts);
    if (rc == HE_OK && out_layout) rc = he_pool_out_layout(p, out_layout);
    if (rc == HE_OK) rc = he_pool_run(c, p, in_cts, out_cts, mode, stream);
    if (rc == HE_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) rc = HE_ECUDA;
    he_pool_destroy(p);
    return rc;
}

extern "C" int he_layout_image(int c, int m, int N, he_layout *out) {
    if (c < 1 || m < 2 || N < 4 || (N & (N - 1)) || !out) { he_set_error("he_layout_image: bad argument"); return HE_EINVAL; }
    Lay L = image_layout(c, m, N);
    if ((long long)L.M * L.M > N && (N % L.M != 0 || L.M % (N / L.M) != 0)) {
        he_set_error("he_layout_image: frame does not tile the shard");
        return HE_EINVAL;
    }
    return to_c(L, out);
}

// ================================================================================ bootstrapping
// ModRaise, CoeffToSlot, EvalMod, SlotToCoeff (the paper restores levels by bootstrapping,
// Sec. 2 and the Bootstrap rows of the Sec. 5 tables; the construction is documented at
// he_boot_create in the header).  The linear levels reuse the raised-basis fused stages of the
// baby-step giant-step convolution: one ModUp of the input, one ModDown per partial sum, one
// ModUp per partial sum and one ModDown for the output.
namespace {
typedef std::complex<double> cplx;
typedef std::map<int, std::vector<cplx>> Diags;          // offset mod N -> values over rows

// Non-zero diagonals of the butterfly stage S_h (inverse: 2 S_h^-1) on N slots.  Row x sits at
// p = x mod 2h of its block, j = p mod h, twiddle exp(2 pi i (5^j mod 8h) / 8h):
//   S_h:       p < h: v[x] + tw v[x+h];   p >= h: v[x-h] - tw v[x]
//   2 S_h^-1:  p < h: v[x] + v[x+h];      p >= h: conj(tw) (v[x-h] - v[x])
Diags stage_diags(int N, int h, bool inverse) {
    std::vector<cplx> tw(h);
    const u64 m = 8ull * (u64)h;
    u64 e = 1;
    for (int j = 0; j < h; j++) {
        tw[j] = std::polar(1.0, 2.0 * M_PI * (double)e / (double)m);
        e = e * 5 % m;
    }
    std::vector<cplx> d0(N), dp(N), dm(N);
    for (int x = 0; x < N; x++) {
        const int p = x % (2 * h);
        const cplx t = tw[p % h];
        if (p < h) {
            d0[x] = 1.0;
            dp[x] = inverse ? cplx(1.0) : t;
        } else {
            d0[x] = inverse ? -std::conj(t) : -t;
            dm[x] = inverse ? std::conj(t) : cplx(1.0);
        }
    }
    Diags D;
    D[0] = d0;
    D[h % N] = dp;
    auto &v = D[(N - h) % N];                             // h = N/2: +h and -h are one diagonal
    if (v.empty()) v = dm;
    else for (int x = 0; x < N; x++) v[x] += dm[x];
    return D;
}

// diagonals of A B (B applied first): diag_d(AB)[x] = sum_e diag_e(A)[x] diag_(d-e)(B)[x+e]
Diags diag_product(const Diags &A, const Diags &B, int N) {
    Diags out;
    for (auto &a : A)
        for (auto &b : B) {
            const int d = (a.first + b.first) % N;
            auto &o = out[d];
            if (o.empty()) o.assign(N, cplx(0.0));
            for (int x = 0; x < N; x++) o[x] += a.second[x] * b.second[(x + a.first) % N];
        }
    for (auto it = out.begin(); it != out.end();) {
        bool nz = false;
        for (auto &v : it->second)
            if (v != cplx(0.0)) { nz = true; break; }
        it = nz ? std::next(it) : out.erase(it);
    }
    return out;
}

// stage counts of the merged levels: logN stages into `levels` groups, the larger ones first
std::vector<int> level_groups(int logN, int levels) {
    std::vector<int> g(levels, logN / levels);
    for (int i = 0; i < logN % levels; i++) g[i]++;
    return g;
}

int floor_div(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }
}  // namespace

// One merged level: offset d = (i b1 + j) u, u = the smallest stage half-length, k = d / u
// taken in [-N/2u, N/2u), i = floor(k / b1), j = k - i b1, b1 the smallest power of two with
// 2 b1 >= k_max - k_min + 1 (two giant steps: a giant partial sum costs a ModUp and a ModDown,
// a baby rotation only a key read).  Partial sum S_i = sum_j rot_(-i b1 u)(diag_d) (.)
// rot_(j u)(x), output sum_i rot_(i b1 u)(S_i).
struct BootLin {
    he_ctx *c = nullptr;
    int stage = 0, idx = 0, level = 0;
    int unit = 1, b1 = 1;
    double gain = 1.0;
    std::vector<int> giants;                      // giant indices, ascending
    std::vector<std::vector<int>> js;             // per giant: baby indices, ascending
    std::vector<std::vector<cplx>> vals;          // per term (giant-major): the rotated diagonal (until encoded)
    size_t terms = 0;
    size_t pw = 0, pe = 0;
    u64 *pts = nullptr, *R = nullptr, *Sb = nullptr, *acc = nullptr;
    FusedStage B, G;
    bool prepared = false;
    size_t n_terms() const { return terms; }
    ~BootLin() { he_free(pts); he_free(R); he_free(Sb); he_free(acc); }
    void amounts(std::set<int> &out) const {
        const int N = c->N;
        for (size_t g = 0; g < giants.size(); g++) {
            const int a = ((giants[g] * b1 * unit) % N + N) % N;
            if (a) out.insert(a);
            for (int j : js[g])
                if ((j * unit) % N) out.insert((j * unit) % N);
        }
    }
};

static int boot_lin_plan(he_ctx *c, BootLin &L, const std::vector<int> &hs, const Diags &D) {
    const int N = c->N;
    L.unit = *std::min_element(hs.begin(), hs.end());
    const int span = N / L.unit;
    std::map<int, const std::vector<cplx> *> ks;
    for (auto &d : D) {
        int k = d.first / L.unit;
        if (2 * k >= span) k -= span;
        ks[k] = &d.second;
    }
    const int kmin = ks.begin()->first, kmax = ks.rbegin()->first;
    L.b1 = 1;
    while (2 * L.b1 < kmax - kmin + 1) L.b1 *= 2;
    std::map<int, std::map<int, const std::vector<cplx> *>> by;
    for (auto &kv : ks) {
        const int i = floor_div(kv.first, L.b1);
        by[i][kv.first - i * L.b1] = kv.second;
    }
    for (auto &gi : by) {
        L.giants.push_back(gi.first);
        L.js.emplace_back();
        const int sh = gi.first * L.b1 * L.unit;          // rot_(-sh): value at x is diag[x - sh]
        for (auto &bj : gi.second) {
            L.js.back().push_back(bj.first);
            const std::vector<cplx> &v = *bj.second;
            std::vector<cplx> r(N);
            for (int x = 0; x < N; x++) r[x] = v[(((x - sh) % N) + N) % N];
            L.vals.push_back(std::move(r));
        }
    }
    L.terms = L.vals.size();
    return HE_OK;
}

// encode the level's diagonals (or take given integers) at scale q_level over Q_level u P
static int boot_lin_upload(he_ctx *c, BootLin &L, const int64_t *given) {
    const size_t n = c->n, T = L.n_terms();
    if (!L.pts) HE_TRY(dev_alloc(&L.pts, T * L.pe));
    std::vector<const double *> none;
    if (given) return upload_plaintexts(c, none, T, 0.0, L.level, L.pts, given, true);
    if (L.vals.size() != T) { he_set_error("bootstrap level: diagonals already released"); return HE_ESTATE; }
    std::vector<int64_t> ints(T * n);
    std::vector<double> re(c->N), im(c->N);
    const double S = (double)c->primes[L.level];
    for (size_t t = 0; t < T; t++) {
        for (int x = 0; x < c->N; x++) {
            re[x] = L.vals[t][x].real();
            im[x] = L.vals[t][x].imag();
        }
        encode_slots_complex(re.data(), im.data(), (int)n, S, ints.data() + t * n);
    }
    return upload_plaintexts(c, none, T, 0.0, L.level, L.pts, ints.data(), true);
}

static int boot_lin_prepare(BootLin &L) {
    if (L.prepared) return HE_OK;
    he_ctx *c = L.c;
    const size_t ng = L.giants.size();
    HE_TRY(dev_alloc(&L.R, 2 * L.pw));
    HE_TRY(dev_alloc(&L.Sb, ng * 2 * L.pw));
    HE_TRY(dev_alloc(&L.acc, 2 * L.pw));
    L.B.c = L.G.c = c;
    L.B.level = L.G.level = L.level;
    L.B.pt_level = L.level;
    char nm[64];
    snprintf(nm, sizeof(nm), "boot %s%d", L.stage ? "stc" : "cts", L.idx);
    L.B.name = std::string(nm) + " baby";
    L.G.name = std::string(nm) + " giant";
    L.B.add_src(L.R, L.pw);
    for (size_t g = 0; g < ng; g++) L.B.add_out(L.Sb + g * 2 * L.pw, L.pw);
    size_t t = 0;
    for (size_t g = 0; g < ng; g++)
        for (int j : L.js[g]) L.B.add_term((int)g, 0, j * L.unit, L.pts + (t++) * L.pe);
    for (size_t g = 0; g < ng; g++) L.G.add_src(L.Sb + g * 2 * L.pw, L.pw);
    L.G.add_out(L.acc, L.pw);
    for (size_t g = 0; g < ng; g++) L.G.add_term(0, (int)g, L.giants[g] * L.b1 * L.unit, HE_PT_ONE);
    HE_TRY(L.B.build());
    HE_TRY(L.G.build());
    L.prepared = true;
    return HE_OK;
}

static int boot_lin_run(he_ctx *c, BootLin &L, const he_ct *in, he_ct *out, cudaStream_t s) {
    if (!in || in->ctx != c || in->level != L.level || !out || out == in) {
        he_set_error("bootstrap linear level: input must sit at level %d", L.level);
        return HE_ELEVEL;
    }
    HE_TRY(boot_lin_prepare(L));
    HE_TRY(k_copy_limbs(L.R, L.pw, in->d, in->pstride, L.pw, 2, s));
    HE_TRY(L.B.run(s));
    HE_TRY(L.G.run(s));
    he_ct t = view(c, L.acc, L.pw, L.level, in->scale * (double)c->primes[L.level]);
    HE_TRY(he_rescale(c, &t, s));
    HE_TRY(ensure_ct(c, out, L.level - 1));
    HE_TRY(k_copy_limbs(out->d, out->pstride, L.acc, L.pw, (size_t)L.level * c->n, 2, s));
    out->scale = t.scale * L.gain;
    return HE_OK;
}

struct he_boot {
    he_ctx *c = nullptr;
    he_boot_config cfg{};
    std::vector<std::unique_ptr<BootLin>> lin[2];     // 0: CoeffToSlot, 1: SlotToCoeff
    std::vector<double> coeffs;
    int depth = 0, evalmod_level = 0, top_stc = 0, out_level = 0;
    he_ct *x = nullptr, *y = nullptr, *cj = nullptr, *re = nullptr, *im = nullptr, *sq = nullptr, *sq2 = nullptr;
    he_ct *m0 = nullptr, *m1 = nullptr, *m2 = nullptr;   // the meta-bootstrap's level-0 input, c1, y / e
    ~he_boot() {
        for (he_ct *t : {x, y, cj, re, im, sq, sq2, m0, m1, m2}) he_ct_free(t);
    }
};

// Chebyshev interpolant at the deg + 1 first-kind nodes of cos(2 pi (K u - 1/4) / 2^r) on [-1, 1]
static void boot_cos_coeffs(int K, int r, int deg, std::vector<double> &c) {
    const int M = deg + 1;
    std::vector<double> f(M);
    for (int k = 0; k < M; k++) {
        const double u = std::cos(M_PI * (k + 0.5) / M);
        f[k] = std::cos(2.0 * M_PI * (K * u - 0.25) / std::ldexp(1.0, r));
    }
    c.assign(M, 0.0);
    for (int j = 0; j < M; j++) {
        double acc = 0;
        for (int k = 0; k < M; k++) acc += f[k] * std::cos(j * M_PI * (k + 0.5) / M);
        c[j] = 2.0 / M * acc;
    }
    c[0] *= 0.5;
}

extern "C" int he_boot_create(he_ctx *c, const he_boot_config *cfg_in, he_boot **out) {
    if (!c || !out) { he_set_error("he_boot_create: null argument"); return HE_EINVAL; }
    *out = nullptr;
    he_boot_config cfg{16, 2, 59, 3, 3};
    if (cfg_in) {
        if (cfg_in->K > 0) cfg.K = cfg_in->K;
        if (cfg_in->double_angle > 0) cfg.double_angle = cfg_in->double_angle;
        if (cfg_in->deg > 0) cfg.deg = cfg_in->deg;
        if (cfg_in->levels_cts > 0) cfg.levels_cts = cfg_in->levels_cts;
        if (cfg_in->levels_stc > 0) cfg.levels_stc = cfg_in->levels_stc;
    }
    const int logN = c->logn - 1;
    if (cfg.deg < 2 || cfg.deg > 255 || cfg.levels_cts > logN || cfg.levels_stc > logN || cfg.double_angle > 16) {
        he_set_error("he_boot_create: bad configuration");
        return HE_EINVAL;
    }
    std::unique_ptr<he_boot> bt(new he_boot());
    bt->c = c;
    bt->cfg = cfg;
    boot_cos_coeffs(cfg.K, cfg.double_angle, cfg.deg, bt->coeffs);
    int k;
    std::vector<int> giants;
    ps_params(cfg.deg, k, giants);
    bt->depth = ps_need(bt->coeffs, k, giants);
    const int L = c->L;
    bt->evalmod_level = L - cfg.levels_cts - 1;
    bt->top_stc = bt->evalmod_level - bt->depth - cfg.double_angle;
    bt->out_level = bt->top_stc - cfg.levels_stc;
    if (bt->out_level < 0) {
        he_set_error("he_boot_create: the bootstrap needs %d levels, the chain has %d",
                     L - bt->out_level, L);
        return HE_ELEVEL;
    }
    const int N = c->N;
    for (int st = 0; st < 2; st++) {
        const int levels = st == 0 ? cfg.levels_cts : cfg.levels_stc;
        std::vector<int> grp = level_groups(logN, levels);
        if (st == 1) std::reverse(grp.begin(), grp.end());
        std::vector<int> hs;                              // CoeffToSlot: N/2 .. 1; SlotToCoeff: 1 .. N/2
        for (int e = 0; e < logN; e++) hs.push_back(st == 0 ? 1 << (logN - 1 - e) : 1 << e);
        size_t pos = 0;
        for (int i = 0; i < levels; i++) {
            std::vector<int> mine(hs.begin() + pos, hs.begin() + pos + grp[i]);
            pos += grp[i];
            Diags D = stage_diags(N, mine[0], st == 0);
            for (size_t a = 1; a < mine.size(); a++) D = diag_product(stage_diags(N, mine[a], st == 0), D, N);
            std::unique_ptr<BootLin> Lv(new BootLin());
            Lv->c = c;
            Lv->stage = st;
            Lv->idx = i;
            Lv->level = st == 0 ? L - i : bt->top_stc - i;
            Lv->gain = st == 0 ? std::ldexp(1.0, (int)mine.size()) : 1.0;
            Lv->pw = (size_t)(Lv->level + 1) * c->n;
            Lv->pe = (size_t)(Lv->level + 1 + c->K) * c->n;
            HE_TRY(boot_lin_plan(c, *Lv, mine, D));
            HE_TRY(boot_lin_upload(c, *Lv, nullptr));
            std::vector<std::vector<cplx>>().swap(Lv->vals);   // encoded: the host copy goes
            bt->lin[st].push_back(std::move(Lv));
        }
    }
    for (he_ct **t : {&bt->x, &bt->y, &bt->cj, &bt->re, &bt->im, &bt->sq, &bt->sq2, &bt->m0, &bt->m1, &bt->m2})
        HE_TRY(he_ct_alloc(c, L, t));
    *out = bt.release();
    return HE_OK;
}

extern "C" void he_boot_destroy(he_boot *bt) {
    if (bt) cudaDeviceSynchronize();
    delete bt;
}

extern "C" int he_boot_rotations(const he_boot *bt, int32_t *amounts, size_t cap) {
    if (!bt) { he_set_error("null argument"); return HE_EINVAL; }
    std::set<int> a;
    for (int st = 0; st < 2; st++)
        for (auto &L : bt->lin[st]) L->amounts(a);
    size_t i = 0;
    for (int v : a) {
        if (amounts && i < cap) amounts[i] = v;
        i++;
    }
    return (int)i;
}

extern "C" int he_boot_info(const he_boot *bt, int *out_level, int *cts_level, int *evalmod_level, int *stc_level,
                            int *keyswitches) {
    if (!bt) { he_set_error("null argument"); return HE_EINVAL; }
    if (out_level) *out_level = bt->out_level;
    if (cts_level) *cts_level = bt->c->L;
    if (evalmod_level) *evalmod_level = bt->evalmod_level;
    if (stc_level) *stc_level = bt->top_stc;
    if (keyswitches) {
        int ks = 1;                                       // the conjugation
        for (int st = 0; st < 2; st++)
            for (auto &L : bt->lin[st]) {
                std::set<int> a;
                for (size_t g = 0; g < L->giants.size(); g++) {
                    for (int j : L->js[g])
                        if ((j * L->unit) % bt->c->N) a.insert(j);
                    if ((L->giants[g] * L->b1 * L->unit) % bt->c->N) ks++;
                }
                ks += (int)a.size();
            }
        int products = 0, dpth = 0;
        he_poly_ps_plan(bt->cfg.deg, &products, &dpth);
        ks += 2 * (products + bt->cfg.double_angle);
        *keyswitches = ks;
    }
    return HE_OK;
}

extern "C" int he_boot_n_plaintexts(const he_boot *bt, int stage, int idx) {
    if (!bt || stage < 0 || stage > 1 || idx < 0 || idx >= (int)bt->lin[stage].size()) {
        he_set_error("he_boot_n_plaintexts: bad argument");
        return HE_EINVAL;
    }
    return (int)bt->lin[stage][idx]->n_terms();
}

extern "C" int he_boot_import_plaintexts(he_boot *bt, int stage, int idx, const int64_t *pts) {
    if (!bt || !pts || stage < 0 || stage > 1 || idx < 0 || idx >= (int)bt->lin[stage].size()) {
        he_set_error("he_boot_import_plaintexts: bad argument");
        return HE_EINVAL;
    }
    BootLin &L = *bt->lin[stage][idx];
    HE_TRY(boot_lin_upload(bt->c, L, pts));
    L.B.invalidate_pk();
    return HE_OK;
}

extern "C" int he_boot_import_coeffs(he_boot *bt, const double *cheb, int deg) {
    if (!bt || !cheb || deg != bt->cfg.deg) { he_set_error("he_boot_import_coeffs: degree must be %d", bt ? bt->cfg.deg : 0); return HE_EINVAL; }
    bt->coeffs.assign(cheb, cheb + deg + 1);
    return HE_OK;
}

extern "C" int he_boot_lintrans(he_ctx *c, he_boot *bt, int stage, int idx, const he_ct *in, he_ct *out, void *stream) {
    if (!c || !bt || bt->c != c || stage < 0 || stage > 1 || idx < 0 || idx >= (int)bt->lin[stage].size()) {
        he_set_error("he_boot_lintrans: bad argument");
        return HE_EINVAL;
    }
    return boot_lin_run(c, *bt->lin[stage][idx], in, out, (cudaStream_t)stream);
}

// An input above level 0 brought to level 0 at scale q_0 / 2^10: dropped to level 1, times the
// integer round((q_0 / 2^10) q_1 / s), rescaled (scale s k / q_1, exact bookkeeping).
static int boot_to_level0(he_ctx *c, const he_ct *in, he_ct *dst, void *stream) {
    HE_TRY(he_ct_copy(dst, in, stream));
    HE_TRY(he_ct_drop_level(dst, 1));
    const double kk = std::nearbyint((double)c->primes[0] / 1024.0 * (double)c->primes[1] / dst->scale);
    if (!(kk >= 1.0)) { he_set_error("bootstrap: input scale %g too large for level 0", dst->scale); return HE_EINVAL; }
    HE_TRY(he_mul_int(c, dst, kk, stream));
    dst->scale = dst->scale * kk;
    return he_rescale(c, dst, stream);
}

extern "C" int he_bootstrap(he_ctx *c, he_boot *bt, const he_ct *in, he_ct *out, void *stream) {
    if (!c || !bt || bt->c != c || !in || !out || in->ctx != c) { he_set_error("he_bootstrap: bad argument"); return HE_EINVAL; }
    if (out->ctx != c || out->cap < bt->out_level) {
        he_set_error("he_bootstrap: output allocated below level %d", bt->out_level);
        return HE_ELEVEL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const double q0 = (double)c->primes[0];
    he_ct *x = bt->x, *y = bt->y;
    if (in->level > 0) {
        HE_TRY(boot_to_level0(c, in, y, stream));
        in = y;
    }
    const double in_scale = in->scale;
    // ModRaise: slots hold t / (q_0 K)  (in may be y here: he_modraise reads limb 0 first)
    HE_TRY(he_modraise(c, in, c->L, x, stream));
    x->scale = q0 * bt->cfg.K;
    // CoeffToSlot
    for (auto &L : bt->lin[0]) {
        HE_TRY(boot_lin_run(c, *L, x, y, s));
        std::swap(x, y);
    }
    // retarget to about Delta / 2 (exact scale bookkeeping)
    {
        const double kk = std::nearbyint(c->pr.scale / 2.0 * (double)c->primes[x->level] / x->scale);
        if (!(kk >= 1.0)) { he_set_error("bootstrap: scale %g too large to retarget", x->scale); return HE_EINVAL; }
        HE_TRY(he_mul_int(c, x, kk, stream));
        x->scale = x->scale * kk;
        HE_TRY(he_rescale(c, x, stream));
    }
    // split: re = x + conj(x), im = (x - conj(x)) X^(3n/2), both at twice the scale
    HE_TRY(he_conjugate(c, x, bt->cj, stream));
    HE_TRY(he_ct_copy(bt->re, x, stream));
    HE_TRY(he_add(c, bt->re, bt->cj, stream));
    bt->re->scale = x->scale * 2.0;
    HE_TRY(he_ct_copy(bt->im, x, stream));
    HE_TRY(he_sub(c, bt->im, bt->cj, stream));
    HE_TRY(he_mul_monomial(c, bt->im, 3 * (int64_t)c->n / 2, stream));
    bt->im->scale = x->scale * 2.0;
    // EvalMod: cosine by Paterson-Stockmeyer, then r double angles
    he_ct *pair[2] = {bt->re, bt->im};
    const double tg[2] = {c->pr.scale, c->pr.scale};
    HE_TRY(he_poly_eval_ps_many(c, pair, 2, bt->coeffs.data(), bt->cfg.deg, tg, stream));
    he_ct *sq[2] = {bt->sq, bt->sq2};
    for (int r = 0; r < bt->cfg.double_angle; r++) {
        // both halves' squares in one batched relinearisation (the bits of he_mul_relin)
        HE_TRY(relin_batch(c, {pair[0], pair[1]}, {pair[0], pair[1]}, {sq[0], sq[1]}, s));
        for (int h = 0; h < 2; h++) {
            HE_TRY(he_mul_int(c, sq[h], 2.0, stream));
            HE_TRY(he_add_const_int(c, sq[h], -std::nearbyint(sq[h]->scale), stream));
            std::swap(pair[h], sq[h]);
        }
    }
    bt->re = pair[0];                                     // a permutation of the plan's four buffers
    bt->im = pair[1];
    bt->sq = sq[0];
    bt->sq2 = sq[1];
    // recombine: re + i im, slots m / Delta_in
    HE_TRY(he_mul_monomial(c, bt->im, (int64_t)c->n / 2, stream));
    HE_TRY(he_ct_copy(x, bt->re, stream));
    HE_TRY(he_add(c, x, bt->im, stream));
    x->scale = x->scale * (2.0 * M_PI * in_scale / q0);
    {
        // back to about Delta without a level: times the integer round(Delta / s)
        const double kk = std::nearbyint(c->pr.scale / x->scale);
        if (kk > 1.0) {
            HE_TRY(he_mul_int(c, x, kk, stream));
            x->scale = x->scale * kk;
        }
    }
    // SlotToCoeff
    for (auto &L : bt->lin[1]) {
        HE_TRY(boot_lin_run(c, *L, x, y, s));
        std::swap(x, y);
    }
    HE_TRY(ensure_ct(c, out, x->level));
    HE_TRY(he_ct_copy(out, x, stream));
    out->scale = x->scale;
    return HE_OK;
}

// Bootstrapping with its own error removed once more (the paper's Appendix on precision and
// bootstrapping noise, MetaBTS): c1 = bootstrap(ct); y = c1 brought back to level 0 at ct's
// scale (dropped to level 1, times round(s0 q_1 / s), rescaled, read at s0); e = (y - ct) 2^kb
// encrypts the bootstrap's error 2^kb times larger; f = bootstrap(e) with its scale times 2^kb;
// g = f times round(s1 q_lv / s_f), rescaled, read at c1's scale; out = c1 (dropped) - g, one
// level below the bootstrap's output.
extern "C" int he_bootstrap_meta(he_ctx *c, he_boot *bt, const he_ct *in, int kb, he_ct *out, void *stream) {
    if (!c || !bt || bt->c != c || !in || !out || in->ctx != c || kb < 0 || kb > 30) {
        he_set_error("he_bootstrap_meta: bad argument");
        return HE_EINVAL;
    }
    if (bt->out_level < 1 || out->ctx != c || out->cap < bt->out_level) {
        he_set_error("he_bootstrap_meta: needs the bootstrap's output level (%d) and one more", bt->out_level);
        return HE_ELEVEL;
    }
    he_ct *ct0 = bt->m0, *c1 = bt->m1, *y = bt->m2;
    if (in->level > 0) HE_TRY(boot_to_level0(c, in, ct0, stream));
    else HE_TRY(he_ct_copy(ct0, in, stream));
    const double s0 = ct0->scale;
    HE_TRY(he_bootstrap(c, bt, ct0, c1, stream));
    // y = c1 at level 0, read at s0
    HE_TRY(he_ct_copy(y, c1, stream));
    HE_TRY(he_ct_drop_level(y, 1));
    const double k = std::nearbyint(s0 * (double)c->primes[1] / y->scale);
    if (!(k >= 1.0)) { he_set_error("he_bootstrap_meta: scale out of range"); return HE_EINVAL; }
    HE_TRY(he_mul_int(c, y, k, stream));
    y->scale = y->scale * k;
    HE_TRY(he_rescale(c, y, stream));
    y->scale = s0;
    // e = (y - ct) 2^kb
    HE_TRY(he_sub(c, y, ct0, stream));
    HE_TRY(he_mul_int(c, y, std::ldexp(1.0, kb), stream));
    // f = bootstrap(e), value E (its scale times 2^kb)
    HE_TRY(he_bootstrap(c, bt, y, out, stream));
    out->scale = out->scale * std::ldexp(1.0, kb);
    const int lv = out->level;
    const double kf = std::nearbyint(c1->scale * (double)c->primes[lv] / out->scale);
    if (!(kf >= 1.0)) { he_set_error("he_bootstrap_meta: scale out of range"); return HE_EINVAL; }
    HE_TRY(he_mul_int(c, out, kf, stream));
    out->scale = out->scale * kf;
    HE_TRY(he_rescale(c, out, stream));
    // out = c1 (dropped to lv - 1) - g
    HE_TRY(he_ct_drop_level(c1, lv - 1));
    HE_TRY(he_sub(c, c1, out, stream));
    HE_TRY(he_ct_copy(out, c1, stream));
    return HE_OK;
}
