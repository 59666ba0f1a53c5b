// api_tt.cu -- the C ABI of the TT algebra around the cross evaluation:
// TT-rounding of batched TT sums (weno_tt_round), batched maxvol (weno_maxvol)
// and the fixed-rank TT-cross sweep (weno_tt_cross).  Host orchestration only;
// the kernels are in k_tt.cu, k_maxvol.cu and k_cross_drv.cu.
#include "api_ctx.h"

using namespace wg;

// ------------------------------------------------------------ TT-rounding
// weno_tt_round: round(sum_t c_t X_t, eps) for a batch of 3D TTs (Sec. 3
// "TT-rounding"; the stages of Eq. tt-ssprk3 are such sums).  Phase 1
// (right-to-left orthogonalisation and the first truncated SVD) and phase 2
// (the second SVD) end with a host read of the ranks they chose, which size
// the launches that follow.

namespace {

struct QRPlan {
    long long m = 0;
    int k = 0, b = 32, C = 1, sub = 1, top_sub = 0;
    long long chunk_rows = 0;
    double *A = nullptr, *tau = nullptr, *Rc = nullptr, *tau_top = nullptr, *T = nullptr;
};

// Chunking of an m x k QR: sub-blocks of b >= k rows, at most 16 per chunk,
// every chunk at least k rows long when there are several.
void qr_plan(QRPlan &q, long long m, int k)
{
    q.m = m;
    q.k = k;
    q.b = k <= 32 ? 32 : (k + 31) / 32 * 32;
    int C = (int)std::max(1LL, (m + 16LL * q.b - 1) / (16LL * q.b));
    for (;; --C) {
        const long long cr = (m + C - 1) / C;
        if (C == 1 || (cr >= k && m - (long long)(C - 1) * cr >= k)) {
            q.C = C;
            q.chunk_rows = std::max(1LL, cr);
            break;
        }
    }
    q.sub = (int)((q.chunk_rows + q.b - 1) / q.b);
    q.top_sub = q.C > 1 ? (int)(((long long)q.C * k + q.b - 1) / q.b) : 0;
}

struct Bump {  // counts (base == nullptr) or hands out 256-byte aligned pieces
    char *base = nullptr;
    size_t off = 0;
    template <class T> T *take(size_t n)
    {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += sizeof(T) * n;
        return p;
    }
};

void qr_take(Bump &bp, QRPlan &q)
{
    q.tau = bp.take<double>((size_t)q.C * q.sub * q.k);
    q.Rc = bp.take<double>((size_t)q.C * q.k * q.k);
    if (q.C > 1) {
        q.tau_top = bp.take<double>((size_t)q.top_sub * q.k);
        q.T = bp.take<double>((size_t)q.k * q.k);
    } else {
        q.T = q.Rc;
    }
}

struct TTPlan {
    int n[3] = {0, 0, 0};
    int R1 = 0, R2 = 0, k3 = 0, k2 = 0, kc = 0, ke = 0;
    long long mB = 0;
    double *C1 = nullptr, *MA = nullptr, *MB = nullptr, *MC = nullptr, *ME = nullptr;
    QRPlan qa, qb, qc, qe, qe_max;
    double *VC = nullptr, *WC = nullptr, *svC = nullptr, *VE = nullptr, *WE = nullptr, *svE = nullptr;
    double *delta = nullptr;
    double *XSa = nullptr, *XSb = nullptr, *XSc = nullptr, *XSe = nullptr;
    int r1 = 0, r2 = 0;
};

}  // namespace

// Factor every plan (leaf chunks, then the stacked chunk R factors).
static int tt_factor(weno_ctx *h, std::vector<QRPlan *> &ps, QRDesc *dev)
{
    const int n = (int)ps.size();
    std::vector<QRDesc> leaf(n), top(n);
    int maxC = 1, maxk = 1, maxb = 32;
    bool any_top = false;
    for (int i = 0; i < n; ++i) {
        const QRPlan &q = *ps[i];
        leaf[i] = QRDesc{q.A, q.m, q.k, q.k, q.b, q.C, q.chunk_rows, q.sub, q.tau, q.Rc};
        top[i] = QRDesc{q.Rc, q.C > 1 ? (long long)q.C * q.k : 0, q.k, q.k, q.b, 1, (long long)q.C * q.k,
                        q.top_sub, q.tau_top, q.T};
        maxC = std::max(maxC, q.C);
        maxk = std::max(maxk, q.k);
        maxb = std::max(maxb, q.b);
        any_top |= q.C > 1;
    }
    const size_t smem = qr_factor_smem(maxk, maxb);
    CK(h, cudaMemcpyAsync(dev, leaf.data(), sizeof(QRDesc) * n, cudaMemcpyHostToDevice, h->stream));
    CK(h, launch(h, 0, h->stream, [&] { return launch_qr_factor(dev, n, maxC, smem, h->stream); }));
    if (any_top) {
        CK(h, cudaMemcpyAsync(dev + n, top.data(), sizeof(QRDesc) * n, cudaMemcpyHostToDevice, h->stream));
        CK(h, launch(h, 0, h->stream, [&] { return launch_qr_factor(dev + n, n, 1, smem, h->stream); }));
    }
    return WENO_OK;
}

struct ApplyReq {  // Q [X; 0] of one plan into an output row map
    const QRPlan *q;
    const double *X;
    int ldx, p;
    double *XS;  // stack of the chunks' top rows (C > 1)
    double *out;
    long long P, sP, sQ, sC;
};

static int tt_apply(weno_ctx *h, std::vector<ApplyReq> &rs, QApplyDesc *dev)
{
    const int n = (int)rs.size();
    std::vector<QApplyDesc> leaf(n), top(n);
    int maxC = 1, maxk = 1, maxb = 32, maxp = 1;
    bool any_top = false;
    for (int i = 0; i < n; ++i) {
        const ApplyReq &r = rs[i];
        const QRPlan &q = *r.q;
        const bool two = q.C > 1;
        const long long mt = (long long)q.C * q.k;
        top[i] = QApplyDesc{q.Rc, q.tau_top, two ? mt : 0, q.k, q.k, q.b, 1, mt, q.top_sub, r.X, 0, r.ldx, r.p,
                            r.XS, mt, r.p, 0, 1};
        leaf[i] = QApplyDesc{q.A, q.tau, q.m, q.k, q.k, q.b, q.C, q.chunk_rows, q.sub, two ? r.XS : r.X,
                             two ? (long long)q.k * r.p : 0, two ? r.p : r.ldx, r.p, r.out, r.P, r.sP, r.sQ, r.sC};
        maxC = std::max(maxC, q.C);
        maxk = std::max(maxk, q.k);
        maxb = std::max(maxb, q.b);
        maxp = std::max(maxp, r.p);
        any_top |= two;
    }
    const size_t smem = qr_apply_smem(maxk, maxb, maxp);
    if (any_top) {
        CK(h, cudaMemcpyAsync(dev + n, top.data(), sizeof(QApplyDesc) * n, cudaMemcpyHostToDevice, h->stream));
        CK(h, launch(h, 0, h->stream, [&] { return launch_qr_apply(dev + n, n, 1, smem, h->stream); }));
    }
    CK(h, cudaMemcpyAsync(dev, leaf.data(), sizeof(QApplyDesc) * n, cudaMemcpyHostToDevice, h->stream));
    CK(h, launch(h, 0, h->stream, [&] { return launch_qr_apply(dev, n, maxC, smem, h->stream); }));
    return WENO_OK;
}

static int tt_svd(weno_ctx *h, std::vector<SvdDesc> &ds, SvdDesc *dev)
{
    const int n = (int)ds.size();
    int maxpk = 1, maxq = 1;
    for (auto &d : ds) {
        maxpk = std::max(maxpk, d.pk);
        maxq = std::max(maxq, d.q);
    }
    const size_t smem = svd_smem(maxpk, maxq);
    CK(h, cudaMemcpyAsync(dev, ds.data(), sizeof(SvdDesc) * n, cudaMemcpyHostToDevice, h->stream));
    CK(h, launch(h, 1, h->stream, [&] { return launch_svd_jacobi(dev, n, smem, h->stream); }));
    return WENO_OK;
}

extern "C" int weno_tt_round(weno_handle h, weno_tt_round_problem *probs, int32_t n_probs, double eps_tt)
{
    if (!h) return WENO_ERR_ARG;
    if (!probs || n_probs < 1 || n_probs > 65535) return fail(h, WENO_ERR_ARG, "weno_tt_round: need 1..65535 problems");
    if (!(eps_tt >= 0.0)) return fail(h, WENO_ERR_ARG, "weno_tt_round: need eps_tt >= 0");
    const int np = n_probs;
    std::vector<TTPlan> pl(np);
    std::vector<TTSumDesc> sd(np);
    for (int i = 0; i < np; ++i) {
        const weno_tt_round_problem &P = probs[i];
        TTPlan &t = pl[i];
        TTSumDesc &s = sd[i];
        if (P.n_terms < 1 || P.n_terms > WENO_TT_MAX_TERMS) return fail(h, WENO_ERR_ARG, "weno_tt_round: 1..4 terms");
        s.nt = P.n_terms;
        for (int m = 0; m < 3; ++m) t.n[m] = s.n[m] = P.term[0].n[m];
        int a = 0, b = 0;
        for (int k = 0; k < P.n_terms; ++k) {
            const weno_tt3 &X = P.term[k];
            for (int m = 0; m < 3; ++m) {
                if (X.n[m] != t.n[m] || X.n[m] < 1 || X.n[m] > (1 << 20))
                    return fail(h, WENO_ERR_ARG, "weno_tt_round: terms need equal mode sizes in 1..2^20");
                if (!X.core[m]) return fail(h, WENO_ERR_ARG, "weno_tt_round: null core");
                s.core[k][m] = X.core[m];
            }
            if (X.r[0] < 1 || X.r[1] < 1) return fail(h, WENO_ERR_ARG, "weno_tt_round: ranks must be >= 1");
            s.a0[k] = a;
            s.b0[k] = b;
            s.r1[k] = X.r[0];
            s.r2[k] = X.r[1];
            s.coef[k] = P.coef[k];
            a += X.r[0];
            b += X.r[1];
        }
        if (a > TT_KMAX || b > TT_KMAX)
            return fail(h, WENO_ERR_UNSUPPORTED, "weno_tt_round: the ranks of a sum may add up to 96 at most");
        for (int m = 0; m < 3; ++m)
            if (!P.out.core[m]) return fail(h, WENO_ERR_ARG, "weno_tt_round: null output core");
        t.R1 = s.R1 = a;
        t.R2 = s.R2 = b;
        t.k3 = s.k3 = std::min(t.n[2], t.R2);
        t.mB = (long long)t.n[1] * t.k3;
        t.k2 = (int)std::min<long long>(t.mB, t.R1);
        t.kc = std::min(t.n[0], t.k2);
        qr_plan(t.qa, t.n[2], t.R2);
        qr_plan(t.qb, t.mB, t.R1);
        qr_plan(t.qc, t.n[0], t.k2);
        qr_plan(t.qe_max, (long long)t.kc * t.n[1], t.k3);
        t.ke = (int)std::min<long long>((long long)t.kc * t.n[1], t.k3);
    }
    // scratch: descriptors, ranks, then per problem matrices and QR data
    const int NDESC = 24;
    const size_t dsz = std::max({sizeof(QRDesc), sizeof(QApplyDesc), sizeof(SvdDesc), sizeof(TTSumDesc), sizeof(GemmDesc)});
    auto layout = [&](Bump &bp) -> char * {
        char *desc = bp.take<char>(dsz * NDESC * (size_t)np);
        for (auto &t : pl) {
            t.C1 = bp.take<double>((size_t)t.n[0] * t.R1);
            t.MA = bp.take<double>((size_t)t.n[2] * t.R2);
            t.MB = bp.take<double>((size_t)t.mB * t.R1);
            t.MC = bp.take<double>((size_t)t.n[0] * t.k2);
            t.ME = bp.take<double>((size_t)t.kc * t.n[1] * t.k3);
            qr_take(bp, t.qa);
            qr_take(bp, t.qb);
            qr_take(bp, t.qc);
            qr_take(bp, t.qe_max);
            t.VC = bp.take<double>((size_t)t.kc * t.kc);
            t.WC = bp.take<double>((size_t)t.k2 * t.kc);
            t.svC = bp.take<double>(t.kc);
            t.VE = bp.take<double>((size_t)t.ke * t.ke);
            t.WE = bp.take<double>((size_t)t.k3 * t.ke);
            t.svE = bp.take<double>(t.ke);
            t.delta = bp.take<double>(2);
            t.XSa = bp.take<double>((size_t)t.qa.C * t.qa.k * t.ke);
            t.XSb = bp.take<double>((size_t)t.qb.C * t.qb.k * t.kc);
            t.XSc = bp.take<double>((size_t)t.qc.C * t.qc.k * t.kc);
            t.XSe = bp.take<double>((size_t)t.qe_max.C * t.qe_max.k * t.ke);
        }
        return desc;
    };
    Bump count;
    layout(count);
    const size_t rank_off = (count.off + 255) & ~size_t(255);
    const size_t bytes = rank_off + sizeof(int) * 2 * (size_t)np;
    if (bytes > h->tbuf_bytes) {
        CK(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->tbuf);
        h->tbuf = nullptr;
        h->tbuf_bytes = 0;
        CK(h, cudaMalloc(&h->tbuf, bytes));
        h->tbuf_bytes = bytes;
    }
    Bump bp;
    bp.base = (char *)h->tbuf;
    char *desc = layout(bp);
    int *ranks = (int *)((char *)h->tbuf + rank_off);
    int slot = 0;
    auto next_desc = [&]() { return desc + dsz * (size_t)np * (slot++); };

    for (int i = 0; i < np; ++i) {
        TTPlan &t = pl[i];
        sd[i].C1 = t.C1;
        sd[i].MA = t.MA;
        sd[i].MB = t.MB;
        sd[i].TA = t.qa.T;
        t.qa.A = t.MA;
        t.qb.A = t.MB;
        t.qc.A = t.MC;
        t.qe_max.A = t.ME;
    }
    // ---- phase 1: sum unfoldings; QR of the last core; middle core times TA^T; QR; first core; QR; SVD
    {
        TTSumDesc *d = (TTSumDesc *)next_desc();
        CK(h, cudaMemcpyAsync(d, sd.data(), sizeof(TTSumDesc) * np, cudaMemcpyHostToDevice, h->stream));
        CK(h, launch(h, 1, h->stream, [&] { return launch_tt_build(d, np, h->stream); }));
        std::vector<QRPlan *> ps;
        for (auto &t : pl) ps.push_back(&t.qa);
        int r = tt_factor(h, ps, (QRDesc *)next_desc());
        if (r) return r;
        ++slot;
        CK(h, launch(h, 1, h->stream, [&] { return launch_tt_contract(d, np, h->stream); }));
        ps.clear();
        for (auto &t : pl) ps.push_back(&t.qb);
        if ((r = tt_factor(h, ps, (QRDesc *)next_desc()))) return r;
        ++slot;
        std::vector<GemmDesc> gd(np);
        for (int i = 0; i < np; ++i)
            gd[i] = GemmDesc{pl[i].C1, pl[i].qb.T, pl[i].MC, pl[i].n[0], pl[i].k2, pl[i].R1};
        GemmDesc *gdev = (GemmDesc *)next_desc();
        CK(h, cudaMemcpyAsync(gdev, gd.data(), sizeof(GemmDesc) * np, cudaMemcpyHostToDevice, h->stream));
        CK(h, launch(h, 1, h->stream, [&] { return launch_tt_gemm_tr(gdev, np, h->stream); }));
        ps.clear();
        for (auto &t : pl) ps.push_back(&t.qc);
        if ((r = tt_factor(h, ps, (QRDesc *)next_desc()))) return r;
        ++slot;
        std::vector<SvdDesc> sv(np);
        for (int i = 0; i < np; ++i) {
            TTPlan &t = pl[i];
            sv[i] = SvdDesc{t.qc.T, t.k2, t.kc, t.k2, eps_tt, 1, t.delta, ranks + 2 * i, t.kc, t.svC, t.VC, t.WC, t.kc};
        }
        if ((r = tt_svd(h, sv, (SvdDesc *)next_desc()))) return r;
    }
    std::vector<int> rk(2 * np);
    CK(h, cudaMemcpyAsync(rk.data(), ranks, sizeof(int) * 2 * np, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (int i = 0; i < np; ++i) {
        TTPlan &t = pl[i];
        t.r1 = rk[2 * i];
        if (t.r1 < 1 || t.r1 > t.kc) return fail(h, WENO_ERR_CUDA, "weno_tt_round: device returned a bad rank");
        if (probs[i].cap[0] < (long long)t.n[0] * t.r1)
            return fail(h, WENO_ERR_ARG, "weno_tt_round: output core 1 capacity too small");
        t.qe = t.qe_max;
        qr_plan(t.qe, (long long)t.r1 * t.n[1], t.k3);
        t.qe.A = t.ME;
        t.qe.tau = t.qe_max.tau;
        t.qe.Rc = t.qe_max.Rc;
        t.qe.tau_top = t.qe_max.tau_top;
        t.qe.T = t.qe.C > 1 ? t.qe_max.T : t.qe.Rc;
    }
    // ---- phase 2: first output core; the middle core into the (r1 n2) x k3 unfolding; QR; SVD
    {
        std::vector<ApplyReq> ar(np);
        for (int i = 0; i < np; ++i) {
            TTPlan &t = pl[i];
            ar[i] = ApplyReq{&t.qc, t.VC, t.kc, t.r1, t.XSc, probs[i].out.core[0], t.n[0], t.r1, 0, 1};
        }
        int r = tt_apply(h, ar, (QApplyDesc *)next_desc());
        if (r) return r;
        ++slot;
        for (int i = 0; i < np; ++i) {
            TTPlan &t = pl[i];
            ar[i] = ApplyReq{&t.qb, t.WC, t.kc, t.r1, t.XSb, t.ME, t.mB, 1, 0, t.mB};
        }
        if ((r = tt_apply(h, ar, (QApplyDesc *)next_desc()))) return r;
        ++slot;
        std::vector<QRPlan *> ps;
        for (auto &t : pl) ps.push_back(&t.qe);
        if ((r = tt_factor(h, ps, (QRDesc *)next_desc()))) return r;
        ++slot;
        std::vector<SvdDesc> sv(np);
        for (int i = 0; i < np; ++i) {
            TTPlan &t = pl[i];
            const int pk = (int)std::min<long long>((long long)t.r1 * t.n[1], t.k3);
            sv[i] = SvdDesc{t.qe.T, t.k3, pk, t.k3, eps_tt, 0, t.delta, ranks + 2 * i + 1, pk, t.svE, t.VE, t.WE, t.ke};
        }
        if ((r = tt_svd(h, sv, (SvdDesc *)next_desc()))) return r;
    }
    std::vector<double> norms(2 * np);
    CK(h, cudaMemcpyAsync(rk.data(), ranks, sizeof(int) * 2 * np, cudaMemcpyDeviceToHost, h->stream));
    for (int i = 0; i < np; ++i)
        CK(h, cudaMemcpyAsync(&norms[2 * i], pl[i].delta, sizeof(double) * 2, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (int i = 0; i < np; ++i) {
        TTPlan &t = pl[i];
        t.r2 = rk[2 * i + 1];
        if (t.r2 < 1 || t.r2 > t.ke) return fail(h, WENO_ERR_CUDA, "weno_tt_round: device returned a bad rank");
        if (probs[i].cap[1] < (long long)t.n[1] * t.r1 * t.r2 || probs[i].cap[2] < (long long)t.n[2] * t.r2)
            return fail(h, WENO_ERR_ARG, "weno_tt_round: output core 2 or 3 capacity too small");
    }
    // ---- phase 3: middle and last output cores
    {
        std::vector<ApplyReq> ar(np);
        for (int i = 0; i < np; ++i) {
            TTPlan &t = pl[i];
            ar[i] = ApplyReq{&t.qe, t.VE, t.ke, t.r2, t.XSe, probs[i].out.core[1], t.n[1], (long long)t.r1 * t.r2,
                             t.r2, 1};
        }
        int r = tt_apply(h, ar, (QApplyDesc *)next_desc());
        if (r) return r;
        ++slot;
        for (int i = 0; i < np; ++i) {
            TTPlan &t = pl[i];
            ar[i] = ApplyReq{&t.qa, t.WE, t.ke, t.r2, t.XSa, probs[i].out.core[2], t.n[2], t.r2, 0, 1};
        }
        if ((r = tt_apply(h, ar, (QApplyDesc *)next_desc()))) return r;
        ++slot;
    }
    for (int i = 0; i < np; ++i) {
        weno_tt3 &o = probs[i].out;
        for (int m = 0; m < 3; ++m) o.n[m] = pl[i].n[m];
        o.r[0] = pl[i].r1;
        o.r[1] = pl[i].r2;
        probs[i].norm = norms[2 * i + 1];
    }
    return WENO_OK;
}

// ------------------------------------------------------------------ maxvol
extern "C" int weno_maxvol(weno_handle h, const weno_maxvol_problem *probs, int32_t n_probs, double delta,
                           int32_t max_iters, int32_t *swaps)
{
    if (!h) return WENO_ERR_ARG;
    if (!probs || n_probs < 1 || n_probs > 65535) return fail(h, WENO_ERR_ARG, "weno_maxvol: need 1..65535 matrices");
    if (!(delta >= 0.0) || max_iters < 0) return fail(h, WENO_ERR_ARG, "weno_maxvol: need delta >= 0, max_iters >= 0");
    std::vector<MaxvolDesc> ds(n_probs);
    size_t w_total = 0;
    int max_r = 1;
    for (int i = 0; i < n_probs; ++i) {
        const weno_maxvol_problem &P = probs[i];
        if (P.r < 1 || P.r > MV_RMAX || P.n < P.r || P.n > MV_NMAX || !P.A || !P.B || !P.idx)
            return fail(h, WENO_ERR_ARG, "weno_maxvol: need 1 <= r <= 64, r <= n <= 65536 and non-null A, B, idx");
        w_total += (((size_t)P.n * P.r + 31) & ~size_t(31)) + (((size_t)P.r * P.r + 31) & ~size_t(31));
        max_r = std::max(max_r, (int)P.r);
    }
    const size_t off_desc = 0;
    const size_t off_int = (sizeof(MaxvolDesc) * n_probs + 255) & ~size_t(255);
    const size_t off_w = (off_int + sizeof(int) * 2 * n_probs + 255) & ~size_t(255);
    int r = grow(h, &h->mbuf, &h->mbuf_bytes, off_w + sizeof(double) * w_total);
    if (r) return r;
    char *base = (char *)h->mbuf;
    int *ints = (int *)(base + off_int);
    double *w = (double *)(base + off_w);
    for (int i = 0; i < n_probs; ++i) {
        const weno_maxvol_problem &P = probs[i];
        double *linv = w + (((size_t)P.n * P.r + 31) & ~size_t(31));
        ds[i] = MaxvolDesc{P.A, P.B, w, linv, P.idx, ints + 2 * i, ints + 2 * i + 1, P.n, P.r};
        w = linv + (((size_t)P.r * P.r + 31) & ~size_t(31));
    }
    maxvol_order(ds.data(), n_probs);
    MaxvolDesc *dd = (MaxvolDesc *)(base + off_desc);
    CK(h, cudaMemcpyAsync(dd, ds.data(), sizeof(MaxvolDesc) * n_probs, cudaMemcpyHostToDevice, h->stream));
    CK(h, launch(h, 1, h->stream, [&] { return launch_maxvol(dd, n_probs, max_r, delta, max_iters, h->stream); },
                 MV_LAUNCHES));
    std::vector<int> st(2 * n_probs);
    CK(h, cudaMemcpyAsync(st.data(), ints, sizeof(int) * 2 * n_probs, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (int i = 0; i < n_probs; ++i) {
        if (st[2 * i]) return fail(h, WENO_ERR_ARG, "weno_maxvol: the pivot rows of a matrix are singular (rank < r)");
        if (swaps) swaps[i] = st[2 * i + 1];
    }
    return WENO_OK;
}

// ---------------------------------------------------------------- TT-cross
// weno_tt_cross: fixed-rank alternating TT-cross of A(i, j, k, f), the flux_dir
// residual contribution of component f of each TT instance (evaluated on
// fibers by weno_cross_eval), with maxvol selecting the index sets.  Every
// step is batched over the instances and runs on the handle's stream without
// a host round trip; the call synchronises once at the end to read maxvol's
// status words.

namespace {
struct XProb {
    int n[3] = {0, 0, 0};
    int r1 = 0, r2 = 0;
    void *outL0 = nullptr, *outL1 = nullptr, *outL2 = nullptr;
    int *right0 = nullptr, *left1 = nullptr, *right1 = nullptr, *left2 = nullptr;
    double *M0 = nullptr, *M1 = nullptr, *MR2 = nullptr, *MR1 = nullptr;
    double *B1 = nullptr, *BR = nullptr, *Wmv = nullptr, *Linv = nullptr;
    int *idx = nullptr;
};
}  // namespace

extern "C" int weno_tt_cross(weno_handle h, const weno_tt_instance *inst, int32_t n_inst, int32_t flux_dir,
                             weno_tt_cross_problem *probs, int32_t sweeps, double delta, int32_t flags)
{
    if (!h) return WENO_ERR_ARG;
    if (!inst || !probs || n_inst < 1 || n_inst > 65535) return fail(h, WENO_ERR_ARG, "weno_tt_cross: need 1..65535 instances");
    if (flux_dir < 0 || flux_dir > 2 || sweeps < 0 || sweeps > 64 || !(delta >= 0.0))
        return fail(h, WENO_ERR_ARG, "weno_tt_cross: need flux_dir 0..2, sweeps 0..64, delta >= 0");
    const bool fp64 = (flags & WENO_CROSS_FP64_CHECK) != 0;
    const size_t esz = fp64 ? sizeof(double) : sizeof(float);
    const int np = n_inst;
    std::vector<XProb> xp(np);
    int max_r = 1;
    for (int i = 0; i < np; ++i) {
        XProb &x = xp[i];
        const weno_tt_cross_problem &P = probs[i];
        for (int m = 0; m < 3; ++m) x.n[m] = inst[i].n[m];
        x.r1 = P.r[0];
        x.r2 = P.r[1];
        const long long n1 = x.n[0], n2 = x.n[1], n3 = x.n[2];
        if (x.r1 < 1 || x.r1 > MV_RMAX || x.r1 > n1 || x.r1 > 5 * n2 * n3 || x.r2 < 1 || x.r2 > MV_RMAX ||
            x.r2 > (long long)x.r1 * n2 || x.r2 > 5 * n3 || x.r1 > n2 * x.r2)
            return fail(h, WENO_ERR_ARG, "weno_tt_cross: need 1 <= r1 <= min(n1, n2 r2, 64), 1 <= r2 <= min(r1 n2, 5 n3, 64)");
        if (!P.J1 || !P.J2 || !P.I1 || !P.I2 || !P.core[0] || !P.core[1] || !P.core[2])
            return fail(h, WENO_ERR_ARG, "weno_tt_cross: null index set or core");
        max_r = std::max({max_r, x.r1, x.r2});
    }
    const int n_mv = 2 * (sweeps + 1) + 2 * sweeps;  // maxvol calls of the whole run
    const int NSLOT = 4;
    const size_t dsz = std::max(sizeof(MaxvolDesc), sizeof(CrossDrvDesc));
    auto layout = [&](Bump &bp) -> char * {
        char *desc = bp.take<char>(dsz * NSLOT * 2 * (size_t)np);
        for (auto &x : xp) {
            const size_t n1 = x.n[0], n2 = x.n[1], n3 = x.n[2], r1 = x.r1, r2 = x.r2;
            x.outL0 = bp.take<char>(esz * 5 * n1 * r1);
            x.outL1 = bp.take<char>(esz * 5 * r1 * n2 * r2);
            x.outL2 = bp.take<char>(esz * 5 * r2 * n3);
            x.right0 = bp.take<int>(2 * r1);
            x.left1 = bp.take<int>(r1);
            x.right1 = bp.take<int>(r2);
            x.left2 = bp.take<int>(2 * r2);
            x.M0 = bp.take<double>(n1 * r1);
            x.M1 = bp.take<double>(r1 * n2 * r2);
            x.MR2 = bp.take<double>(5 * n3 * r2);
            x.MR1 = bp.take<double>(n2 * r2 * r1);
            x.B1 = bp.take<double>(r1 * n2 * r2);
            const size_t mk = std::max({n1 * r1, r1 * n2 * r2, 5 * n3 * r2, n2 * r2 * r1});
            x.BR = bp.take<double>(mk);
            x.Wmv = bp.take<double>(mk);
            x.Linv = bp.take<double>(std::max(r1, r2) * std::max(r1, r2));
            x.idx = bp.take<int>(std::max(r1, r2));
        }
        return desc;
    };
    Bump count;
    layout(count);
    const size_t st_off = (count.off + 255) & ~size_t(255);
    int r = grow(h, &h->cbuf, &h->cbuf_bytes, st_off + sizeof(int) * 2 * (size_t)n_mv * np);
    if (r) return r;
    Bump bp;
    bp.base = (char *)h->cbuf;
    char *desc = layout(bp);
    int *status = (int *)((char *)h->cbuf + st_off);
    auto slot = [&](int k) { return desc + dsz * 2 * (size_t)np * k; };
    CK(h, cudaMemsetAsync(status, 0, sizeof(int) * 2 * (size_t)n_mv * np, h->stream));

    std::vector<CrossDrvDesc> cd(np);
    auto drv = [&](int kind, auto &&fill) -> int {
        for (int i = 0; i < np; ++i) {
            XProb &x = xp[i];
            const weno_tt_cross_problem &P = probs[i];
            CrossDrvDesc &c = cd[i];
            c = CrossDrvDesc{};
            for (int m = 0; m < 3; ++m) c.n[m] = x.n[m];
            c.r1 = x.r1;
            c.r2 = x.r2;
            c.fp64 = fp64 ? 1 : 0;
            c.I1 = P.I1;
            c.I2 = P.I2;
            c.J1 = P.J1;
            c.J2 = P.J2;
            c.idx = x.idx;
            fill(x, P, c);
        }
        CrossDrvDesc *dd = (CrossDrvDesc *)slot(0);
        CK(h, cudaMemcpyAsync(dd, cd.data(), sizeof(CrossDrvDesc) * np, cudaMemcpyHostToDevice, h->stream));
        CK(h, launch(h, 1, h->stream, [&] { return launch_cross_drv(dd, np, kind, h->stream); }));
        return WENO_OK;
    };
    auto evaluate = [&](int mode) -> int {
        std::vector<weno_fiber_set> fs(np);
        for (int i = 0; i < np; ++i) {
            XProb &x = xp[i];
            weno_fiber_set &f = fs[i];
            f = weno_fiber_set{};
            f.instance = i;
            f.mode = mode;
            f.flux_dir = flux_dir;
            if (mode == 0) { f.n_left = 1; f.left = nullptr; f.n_right = x.r1; f.right = x.right0; f.out = x.outL0; }
            if (mode == 1) { f.n_left = x.r1; f.left = x.left1; f.n_right = x.r2; f.right = x.right1; f.out = x.outL1; }
            if (mode == 2) { f.n_left = x.r2; f.left = x.left2; f.n_right = 1; f.right = nullptr; f.out = x.outL2; }
        }
        return weno_cross_eval(h, inst, np, fs.data(), np, fp64 ? WENO_CROSS_FP64_CHECK : 0);
    };
    int mv_call = 0;
    // maxvol on every problem's fiber matrix of this step (rows x cols); no
    // orthogonalisation first: the pivot rows and B = M M[I]^{-1} depend only
    // on M's column space, and B is formed from the elimination's multipliers
    auto select = [&](double *XProb::*Mp, double *XProb::*Bp, bool b_is_core0, auto &&dims) -> int {
        std::vector<MaxvolDesc> md(np);
        int mr = 1;
        for (int i = 0; i < np; ++i) {
            XProb &x = xp[i];
            int rows, cols;
            dims(x, rows, cols);
            double *Bout = b_is_core0 ? probs[i].core[0] : x.*Bp;
            int *st = status + 2 * ((size_t)mv_call * np + i);
            md[i] = MaxvolDesc{x.*Mp, Bout, x.Wmv, x.Linv, x.idx, st, st + 1, rows, cols};
            mr = std::max(mr, cols);
        }
        maxvol_order(md.data(), np);
        MaxvolDesc *dd = (MaxvolDesc *)slot(3);
        CK(h, cudaMemcpyAsync(dd, md.data(), sizeof(MaxvolDesc) * np, cudaMemcpyHostToDevice, h->stream));
        CK(h, launch(h, 1, h->stream, [&] { return launch_maxvol(dd, np, mr, delta, 200, h->stream); }, MV_LAUNCHES));
        ++mv_call;
        return WENO_OK;
    };
    auto dims_l0 = [](const XProb &x, int &m, int &k) { m = x.n[0]; k = x.r1; };
    auto dims_l1 = [](const XProb &x, int &m, int &k) { m = x.r1 * x.n[1]; k = x.r2; };
    auto dims_r2 = [](const XProb &x, int &m, int &k) { m = 5 * x.n[2]; k = x.r2; };
    auto dims_r1 = [](const XProb &x, int &m, int &k) { m = x.n[1] * x.r2; k = x.r1; };
    auto nofill = [](XProb &, const weno_tt_cross_problem &, CrossDrvDesc &) {};
    for (int it = 0; it <= sweeps; ++it) {
        // ---- left to right
        if ((r = drv(XD_PREP_L0, [](XProb &x, const weno_tt_cross_problem &, CrossDrvDesc &c) { c.right = x.right0; })))
            return r;
        if ((r = evaluate(0))) return r;
        if ((r = drv(XD_GATHER_L0, [](XProb &x, const weno_tt_cross_problem &, CrossDrvDesc &c) {
                 c.out = x.outL0;
                 c.M = x.M0;
             })))
            return r;
        if ((r = select(&XProb::M0, &XProb::BR, true, dims_l0))) return r;
        if ((r = drv(XD_UPDATE_L0, nofill))) return r;
        if ((r = drv(XD_PREP_L1, [](XProb &x, const weno_tt_cross_problem &, CrossDrvDesc &c) {
                 c.left = x.left1;
                 c.right = x.right1;
             })))
            return r;
        if ((r = evaluate(1))) return r;
        if ((r = drv(XD_GATHER_L1, [](XProb &x, const weno_tt_cross_problem &, CrossDrvDesc &c) {
                 c.out = x.outL1;
                 c.M = x.M1;
             })))
            return r;
        if ((r = select(&XProb::M1, &XProb::B1, false, dims_l1))) return r;
        if ((r = drv(XD_UPDATE_L1, [](XProb &x, const weno_tt_cross_problem &P, CrossDrvDesc &c) {
                 c.B = x.B1;
                 c.core = P.core[1];
             })))
            return r;
        if ((r = drv(XD_PREP_L2, [](XProb &x, const weno_tt_cross_problem &, CrossDrvDesc &c) { c.left = x.left2; })))
            return r;
        if ((r = evaluate(2))) return r;
        if ((r = drv(XD_GATHER_L2, [](XProb &x, const weno_tt_cross_problem &P, CrossDrvDesc &c) {
                 c.out = x.outL2;
                 c.M = x.MR2;
                 c.core = P.core[2];
             })))
            return r;
        if (it == sweeps) break;
        // ---- right to left
        if ((r = select(&XProb::MR2, &XProb::BR, false, dims_r2))) return r;
        if ((r = drv(XD_UPDATE_R2, nofill))) return r;
        if ((r = drv(XD_PREP_L1, [](XProb &x, const weno_tt_cross_problem &, CrossDrvDesc &c) {
                 c.left = x.left1;
                 c.right = x.right1;
             })))
            return r;
        if ((r = evaluate(1))) return r;
        if ((r = drv(XD_GATHER_R1, [](XProb &x, const weno_tt_cross_problem &, CrossDrvDesc &c) {
                 c.out = x.outL1;
                 c.M = x.MR1;
             })))
            return r;
        if ((r = select(&XProb::MR1, &XProb::BR, false, dims_r1))) return r;
        if ((r = drv(XD_UPDATE_R1, nofill))) return r;
    }
    std::vector<int> st(2 * (size_t)n_mv * np);
    CK(h, cudaMemcpyAsync(st.data(), status, sizeof(int) * st.size(), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (size_t k = 0; k < st.size(); k += 2)
        if (st[k]) return fail(h, WENO_ERR_ARG, "weno_tt_cross: a fiber matrix had rank below the cross rank");
    return WENO_OK;
}
