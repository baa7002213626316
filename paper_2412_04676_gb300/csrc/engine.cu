// engine.cu -- host orchestration of the two-site DMRG iteration on one GB300.
//
// Sec. II.B of arXiv:2412.04676 splits one DMRG iteration at the two-site
// position (b, b+1) into (1) pre-processing: environments of the left block
// (orbitals 0..b-1) and right block (orbitals b+2..L-1) are enlarged by one
// orbital each, O^Lx_c = sum_a W_b[a,c] (x) E^L[a], O^xR_c = sum_e W_{b+1}[c,e]
// (x) E^R[e]; (2) diagonalisation: Davidson on H_eff psi = sum_c O^Lx_c psi
// (O^xR_c)^T; (3) post-processing: per-sector density matrix, global
// selection of at most D states, renormalisation U^T O U of the enlarged
// block's operators and the transformed start vector of the next step
// ("StVec", Sec. IV).  Sec. III.A/B.4 add the asynchronous save of every new
// environment and the load of the next one right after renormalisation.
//
// Every block product runs through one grouped-GEMM launch per phase (FP64
// engine in kernels.cu, BF16x3 tensor-core engine in tc.cu); the host builds
// the task tables from the sector tables (Fig. 4a) and the operator sets of
// Eq. 1 split at every cut (mpo.cpp).
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <chrono>
#include <map>
#include <cmath>
#include <numeric>
#include <random>
#include <thread>

#include "engine.h"

namespace gbd {

double wall_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

void step_mark(Ctx& C, int phase) {
    cudaEvent_t e = nullptr;
    if (C.marks.size() < C.mark_pool.size()) {
        e = C.mark_pool[C.marks.size()];
    } else {
        GBD_CHECK_CUDA(cudaEventCreate(&e));
        C.mark_pool.push_back(e);
    }
    GBD_CHECK_CUDA(cudaEventRecord(e, C.cs));
    C.marks.push_back({phase, e});
}

void step_marks_flush(Ctx& C) {
    for (size_t i = 0; i + 1 < C.marks.size(); ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, C.marks[i].second, C.marks[i + 1].second) == cudaSuccess)
            C.timers[C.marks[i].first] += ms;
    }
    C.marks.clear();
}

// ============================================================== bases
EBasis left_enlarged(const Bond& b) {
    std::map<Q, std::vector<Seg>> m;
    for (int s = 0; s < 4; ++s)
        for (size_t i = 0; i < b.q.size(); ++i) m[b.q[i] + kQS[s]].push_back({s, int(i), 0, b.dim[i]});
    EBasis e;
    for (auto& kv : m) {
        int off = 0;
        for (auto& sg : kv.second) { sg.off = off; off += sg.size; }
        e.q.push_back(kv.first);
        e.dim.push_back(off);
        e.segs.push_back(kv.second);
    }
    return e;
}

EBasis right_enlarged(const Bond& b1) {
    std::map<Q, std::vector<Seg>> m;
    for (int s = 0; s < 4; ++s)
        for (size_t i = 0; i < b1.q.size(); ++i) m[b1.q[i] - kQS[s]].push_back({s, int(i), 0, b1.dim[i]});
    EBasis e;
    for (auto& kv : m) {
        int off = 0;
        for (auto& sg : kv.second) { sg.off = off; off += sg.size; }
        e.q.push_back(kv.first);
        e.dim.push_back(off);
        e.segs.push_back(kv.second);
    }
    return e;
}

namespace {

const Seg* find_seg(const EBasis& e, int qidx, int s) {
    for (const auto& sg : e.segs[qidx])
        if (sg.s == s) return &sg;
    return nullptr;
}

void make_classes(const std::vector<Q>& dq, OpSet& E) {
    std::map<Q, std::vector<int>> g;
    for (size_t i = 0; i < dq.size(); ++i) g[dq[i]].push_back(int(i));
    E.cls.clear();
    E.state_class.assign(dq.size(), -1);
    E.state_layer.assign(dq.size(), -1);
    for (auto& kv : g) {
        OpClass c;
        c.dq = kv.first;
        c.states = kv.second;
        int ci = int(E.cls.size());
        for (size_t l = 0; l < c.states.size(); ++l) {
            E.state_class[c.states[l]] = ci;
            E.state_layer[c.states[l]] = int(l);
        }
        E.cls.push_back(std::move(c));
    }
}

void alloc_env(Ctx& C, OpSet& E) {
    E.layout();
    E.data.alloc_async(size_t(std::max<long long>(E.total, 2)) * sizeof(double), C.cs);
    GBD_CHECK_CUDA(cudaMemsetAsync(E.data.p, 0, size_t(std::max<long long>(E.total, 2)) * sizeof(double), C.cs));
}

// enlarged operator sets live for one position only: from the block cache
void alloc_env_cached(Ctx& C, OpSet& E) {
    E.layout();
    E.data.ensure_cached(size_t(std::max<long long>(E.total, 2)) * sizeof(double), C.cs);
    GBD_CHECK_CUDA(cudaMemsetAsync(E.data.p, 0, size_t(std::max<long long>(E.total, 2)) * sizeof(double), C.cs));
}

std::unique_ptr<OpSet> trivial_env(Ctx& C, int side) {
    auto E = std::make_unique<OpSet>();
    E->side = side;
    E->cut = side == 0 ? 0 : C.L;
    make_classes(C.mpo.dq[E->cut], *E);
    int st = side == 0 ? C.mpo.idxI[0] : C.mpo.idxF[C.L];
    GBD_REQUIRE(st >= 0, GBD_ERR_STATE, "operator sets lack the boundary state");
    int ci = E->state_class[st];
    const Bond& bd = C.bonds[E->cut];
    GBD_REQUIRE(bd.q.size() == 1, GBD_ERR_STATE, "boundary bond must have one sector");
    E->cls[ci].blocks.push_back({0, 0, 1, 1, 0, bd.q[0], bd.q[0]});
    alloc_env(C, *E);
    std::vector<double> v(E->cls[ci].states.size(), 0.0);
    v[E->state_layer[st]] = 1.0;
    E->layout();
    GBD_CHECK_CUDA(cudaMemcpyAsync(E->data.as<double>() + E->cls[ci].blocks[0].off, v.data(), v.size() * sizeof(double),
                                   cudaMemcpyHostToDevice, C.cs));
    GBD_CHECK_CUDA(cudaStreamSynchronize(C.cs));
    return E;
}

}  // namespace

// Links of the enlargement (side, cut k) into the output classes of `out`,
// built on first use (they depend only on the MPO and the classes).
static const EnlLinks& enl_links(Ctx& C, const OpSet& Ein, int side, int k, const OpSet& out) {
    auto& cache = C.enl_links[side];
    if (int(cache.size()) < C.L + 1) cache.resize(C.L + 1);
    EnlLinks& LK = cache[k];
    if (LK.built) return LK;
    const Mpo& M = C.mpo;
    // links between an input class and an output class for one local matrix
    // element (s, t), collected as sparse entries first
    std::map<std::tuple<int, int, int, int>, int> link_id;
    std::vector<EnlLink>& links = LK.links;
    std::vector<std::vector<std::tuple<int, int, double>>> ents;  // (input layer, output layer, value)
    for (const auto& e : M.W[k]) {
        int sin = side == 0 ? e.a : e.c;
        int sout = side == 0 ? e.c : e.a;
        if (sin >= (int)Ein.state_class.size()) continue;
        int ci = Ein.state_class[sin];
        if (ci < 0) continue;
        int li = Ein.state_layer[sin];
        int co = out.state_class[sout], lo = out.state_layer[sout];
        auto key = std::make_tuple(ci, co, e.s, e.t);
        auto it = link_id.find(key);
        int id;
        if (it == link_id.end()) {
            id = int(links.size());
            link_id[key] = id;
            EnlLink L;
            L.ci = ci; L.co = co; L.s = e.s; L.t = e.t;
            links.push_back(std::move(L));
            ents.emplace_back();
        } else {
            id = it->second;
        }
        ents[id].emplace_back(li, lo, e.v);
    }
    // a link whose output layers each take few input layers is a set of
    // scaled copy-sums; the rest (complementary sums over many normal
    // operators) are dense coefficient GEMMs.  With GB300's narrow FP64 pipe
    // a dense GEMM over T_in layers costs T_in FMAs per element, a copy-sum
    // one load per nonzero.
    constexpr int kMaxCopySources = 32;
    LK.sparse.assign(links.size(), 1);
    LK.link_col0.assign(links.size(), -1);
    LK.amax.assign(links.size(), 0);
    long long wtot = 0;
    for (size_t i = 0; i < links.size(); ++i) {
        const int Tin = int(Ein.cls[links[i].ci].states.size());
        const int Tout = int(out.cls[links[i].co].states.size());
        std::vector<int> cnt(Tout, 0);
        for (const auto& x : ents[i]) ++cnt[std::get<1>(x)];
        for (int c = 0; c < Tout; ++c)
            if (cnt[c] > kMaxCopySources) { LK.sparse[i] = 0; break; }
        if (LK.sparse[i]) {
            std::vector<std::vector<std::pair<int, double>>> cs(Tout);
            for (const auto& x : ents[i]) {
                auto& v = cs[std::get<1>(x)];
                bool merged = false;
                for (auto& av : v)
                    if (av.first == std::get<0>(x)) { av.second += std::get<2>(x); merged = true; }
                if (!merged) v.push_back({std::get<0>(x), std::get<2>(x)});
            }
            LK.link_col0[i] = int(LK.ccols.size());
            for (const auto& v : cs) {
                LK.ccols.push_back({int(LK.ccoefs.size()), int(v.size())});
                for (const auto& av : v) {
                    LK.ccoefs.push_back({av.first, av.second});
                    LK.amax[i] = std::max(LK.amax[i], av.first);
                }
            }
        } else {
            links[i].W.assign(size_t(Tin) * Tout, 0.0);
            for (const auto& x : ents[i]) links[i].W[size_t(std::get<0>(x)) * Tout + std::get<1>(x)] += std::get<2>(x);
            links[i].doff = wtot;
            wtot += (long long)links[i].W.size();
        }
        LK.by_cst[std::make_tuple(links[i].co, links[i].s, links[i].t)].push_back(int(i));
    }
    LK.wall.assign(size_t(std::max<long long>(wtot, 1)), 0.0);
    for (size_t i = 0; i < links.size(); ++i)
        if (!LK.sparse[i]) std::copy(links[i].W.begin(), links[i].W.end(), LK.wall.begin() + links[i].doff);
    LK.built = true;
    return LK;
}

// ============================================================== enlargement
// Pre-processing (Sec. II.B step 1): the operators of the enlarged block.
// side 0: Ein = left environment at cut k, output = states of cut k+1 on the
// basis (cut-k bond) + orbital k.  side 1: Ein = right environment at cut
// k+1, output = states of cut k on orbital k + (cut-(k+1) bond).
static void enlarge(Ctx& C, const OpSet& Ein, int side, int k, OpSet& out, EBasis& basis) {
    const double t_host0 = wall_ms();
    const Mpo& M = C.mpo;
    const int out_cut = side == 0 ? k + 1 : k;
    const Bond& bin = C.bonds[side == 0 ? k : k + 1];
    basis = side == 0 ? left_enlarged(bin) : right_enlarged(bin);
    out = OpSet();
    out.side = side;
    out.cut = out_cut;
    make_classes(M.dq[out_cut], out);
    GBD_REQUIRE(Ein.resident(), GBD_ERR_STATE, "environment not resident on the device");

    const EnlLinks& LK = enl_links(C, Ein, side, k, out);
    const std::vector<EnlLink>& links = LK.links;
    const std::vector<char>& sparse = LK.sparse;
    const auto& by_cst = LK.by_cst;
    const double t_links = wall_ms();
    // output blocks and their sub-block tasks
    struct Sub {
        int cls, blk;
        int off_r, off_c, rows, cols;
        std::vector<std::pair<int, int>> src;  // (link, input block)
    };
    std::vector<Sub> subs;
    for (int co = 0; co < (int)out.cls.size(); ++co) {
        OpClass& oc = out.cls[co];
        for (int q2 = 0; q2 < (int)basis.q.size(); ++q2) {
            int q1 = basis.find(basis.q[q2] + oc.dq);
            if (q1 < 0) continue;
            std::vector<Sub> mine;
            for (const auto& sa : basis.segs[q1])
                for (const auto& sb : basis.segs[q2]) {
                    auto it = by_cst.find(std::make_tuple(co, sa.s, sb.s));
                    if (it == by_cst.end()) continue;
                    Sub sub{co, -1, sa.off, sb.off, sa.size, sb.size, {}};
                    for (int li : it->second) {
                        const OpClass& ic = Ein.cls[links[li].ci];
                        int bi = ic.find_block(sb.bq);
                        if (bi < 0 || ic.blocks[bi].qo != sa.bq) continue;
                        sub.src.push_back({li, bi});
                    }
                    if (!sub.src.empty()) mine.push_back(std::move(sub));
                }
            if (mine.empty()) continue;
            int bidx = int(oc.blocks.size());
            oc.blocks.push_back({q1, q2, basis.dim[q1], basis.dim[q2], 0, basis.q[q1], basis.q[q2]});
            for (auto& s : mine) { s.blk = bidx; subs.push_back(std::move(s)); }
        }
    }
    const double t_subs = wall_ms();
    alloc_env_cached(C, out);
    // upload coefficient matrices of the dense links
    const std::vector<double>& wall = LK.wall;
    C.scratch_w.ensure(wall.size() * sizeof(double));
    GBD_CHECK_CUDA(cudaMemcpyAsync(C.scratch_w.p, wall.data(), wall.size() * sizeof(double), cudaMemcpyHostToDevice, C.cs));
    const double* dW = C.scratch_w.as<double>();
    const double* din = Ein.data.as<double>();
    double* dout = out.data.as<double>();
    GemmPlan& P = C.plan_a;
    P.clear();
    std::vector<CopyItem> items;
    std::vector<CopyLink> clinks;
    std::vector<int> clink_amax;  // largest input layer each copy link reads (bounds check)
    // per sparse link, its (input layer, coefficient) lists per output layer
    const std::vector<CopyCol>& ccols = LK.ccols;
    const std::vector<CopyCoef>& ccoefs = LK.ccoefs;
    const std::vector<int>& link_col0 = LK.link_col0;
    int max_tout = 0;
    // mixed form: the dense coefficient GEMMs run on the tensor cores in the
    // sliced form (FP64 GEMMs otherwise)
    const bool tc_env = C.cfg.precision == GBD_MIXED_BF16X3 && C.cfg.mixed_polish == 2;
    std::vector<TcEnlTask> tc_tasks;
    std::vector<TcEnlSeg> tc_segs;
    double tc_flops = 0.0;
    for (const auto& sub : subs) {
        const OpClass& oc = out.cls[sub.cls];
        const OpBlock& ob = oc.blocks[sub.blk];
        int Tout = int(oc.states.size());
        double* dsub = dout + ob.off + (long long)sub.off_r * ob.cols + sub.off_c;
        GemmTask t{};
        t.C = dsub;
        t.ldc = (long long)ob.rows * ob.cols;
        t.ldr = ob.cols;
        t.M = Tout;
        t.N = sub.rows * sub.cols;
        t.ncols = sub.cols;
        t.nbatch = 1;
        t.beta = 0.0;
        std::vector<GemmSeg> segs;
        const int tc_seg0 = int(tc_segs.size());
        std::vector<std::pair<int, const OpBlock*>> sp;  // sparse links of this sub-block
        for (auto& pr : sub.src) {
            const EnlLink& L = links[pr.first];
            const OpClass& ic = Ein.cls[L.ci];
            const OpBlock& ib = ic.blocks[pr.second];
            if (sparse[pr.first]) {
                sp.push_back({pr.first, &ib});
                continue;
            }
            if (tc_env) {
                tc_segs.push_back({dW + L.doff, int(ic.states.size()), Tout, din + ib.off, (long long)ib.rows * ib.cols});
                tc_flops += 2.0 * Tout * double(t.N) * double(ic.states.size());
                continue;
            }
            GemmSeg g{};
            g.A = dW + L.doff;
            g.lda = Tout;
            g.transA = 1;
            g.B = din + ib.off;
            g.ldb = (long long)ib.rows * ib.cols;
            g.transB = 0;
            g.K = int(ic.states.size());
            g.T = 1;
            g.coef = 1.0;
            segs.push_back(g);
        }
        if (int(tc_segs.size()) > tc_seg0)
            tc_tasks.push_back({dsub, t.ldc, t.ldr, t.M, t.N, t.ncols, tc_seg0, int(tc_segs.size()) - tc_seg0});
        if (!segs.empty()) P.add_task(t, segs);
        if (sp.empty()) continue;
        CopyItem it{};
        it.dst = dsub;
        // a sub-block no coefficient GEMM wrote is still zero from the allocation
        it.overwrite = (segs.empty() && int(tc_segs.size()) == tc_seg0) ? 1 : 0;
        it.out_pitch = (long long)ob.rows * ob.cols;
        it.ldr = ob.cols;
        it.rows = sub.rows;
        it.cols = sub.cols;
        it.tout = Tout;
        it.link0 = int(clinks.size());
        for (const auto& lb : sp) {
            clinks.push_back({din + lb.second->off, (long long)lb.second->rows * lb.second->cols, link_col0[lb.first]});
            clink_amax.push_back(LK.amax[lb.first]);
        }
        it.nlink = int(clinks.size()) - it.link0;
        items.push_back(it);
        max_tout = std::max(max_tout, Tout);
    }
    P.check({{C.scratch_w.p, C.scratch_w.bytes}, {Ein.data.p, size_t(Ein.total) * 8}, {out.data.p, size_t(out.total) * 8}},
            "enlarge");
    const double t_items = wall_ms();
    // host-side bounds check of the copies: outputs inside their block arena,
    // inputs inside the environment
    for (const auto& it : items) {
        const double* e = it.dst + (long long)(it.tout - 1) * it.out_pitch + (long long)(it.rows - 1) * it.ldr + it.cols;
        GBD_REQUIRE(it.dst >= dout && e <= dout + out.total, GBD_ERR_STATE, "enlarge: copy outside its block");
        for (int l = it.link0; l < it.link0 + it.nlink; ++l) {
            // every copy of the link reads input layers 0..amax of its block
            const CopyLink& L = clinks[l];
            const double* a = L.src + (long long)clink_amax[l] * L.in_pitch;
            GBD_REQUIRE(L.src >= din && a + (long long)it.rows * it.cols <= din + Ein.total, GBD_ERR_STATE,
                        "enlarge: copy source outside the environment");
        }
    }
    const double t_dev0 = wall_ms();
    C.timers[Ctx::T_ENL_HOST] += t_dev0 - t_host0;
    C.timers[Ctx::T_ENL_H_LINKS] += t_links - t_host0;
    C.timers[Ctx::T_ENL_H_SUBS] += t_subs - t_links;
    C.timers[Ctx::T_ENL_H_ITEMS] += t_items - t_subs;
    C.timers[Ctx::T_ENL_GFLOP] += P.flops * 1e-9;
    P.upload(C.cs);
    P.launch(C.cs);
    if (!tc_tasks.empty()) {
        // bounds of the sliced GEMM outputs and inputs, checked like the FP64 plan's
        for (const auto& tk : tc_tasks) {
            const double* e = tk.C + (long long)(tk.M - 1) * tk.ldc + (long long)((tk.N - 1) / tk.ncols) * tk.ldr +
                              (tk.N - 1) % tk.ncols;
            GBD_REQUIRE(tk.C >= dout && e < dout + out.total, GBD_ERR_STATE, "enlarge: sliced output outside its block");
        }
        for (const auto& sg : tc_segs)
            GBD_REQUIRE(sg.E >= din && sg.E + (long long)sg.Tin * sg.n <= din + Ein.total, GBD_ERR_STATE,
                        "enlarge: sliced input outside the environment");
        tc_enlarge_dense(C, tc_tasks, tc_segs);
        C.timers[Ctx::T_ENL_TC_GFLOP] += tc_flops * 1e-9;
    }
    if (!items.empty()) {
        auto up = [&](DevBuf& d, const void* src, size_t bytes) {  // context buffers, grow-only
            d.ensure(std::max<size_t>(bytes, 16));
            if (bytes) GBD_CHECK_CUDA(cudaMemcpyAsync(d.p, src, bytes, cudaMemcpyHostToDevice, C.cs));
        };
        up(C.scratch_items, items.data(), items.size() * sizeof(CopyItem));
        up(C.scratch_srcs, clinks.data(), clinks.size() * sizeof(CopyLink));
        up(C.scratch_cols, ccols.data(), ccols.size() * sizeof(CopyCol));
        up(C.scratch_coefs, ccoefs.data(), ccoefs.size() * sizeof(CopyCoef));
        copy_sum(C.scratch_items.as<CopyItem>(), int(items.size()), max_tout, C.scratch_srcs.as<CopyLink>(),
                 C.scratch_cols.as<CopyCol>(), C.scratch_coefs.as<CopyCoef>(), C.cs);
    }
    GBD_CHECK_CUDA(cudaStreamSynchronize(C.cs));
    C.timers[Ctx::T_ENL_DEV] += wall_ms() - t_dev0;
}

// ============================================================== renormalisation
// useful flops of the two renormalisation GEMM phases (2 M N K each)
static double renorm_flops(const OpSet& O, const Iso& U, const OpSet& out) {
    (void)O;
    double f = 0.0;
    for (size_t c = 0; c < out.cls.size(); ++c) {
        const double T = double(out.cls[c].states.size());
        for (const auto& nb : out.cls[c].blocks) {
            const double dimO = U.basis.dim[U.basis.find(nb.Qo)], dimI = U.basis.dim[U.basis.find(nb.Qi)];
            f += 2.0 * T * dimO * nb.cols * dimI + 2.0 * T * nb.rows * nb.cols * dimO;
        }
    }
    return f;
}

// Post-processing (Sec. II.B step 3): E_new[t] = U_Q^T O[t] U_Q2 for every
// block of the enlarged operator set whose two sectors are kept.
static void renormalize(Ctx& C, const OpSet& O, const Iso& U, OpSet& out) {
    const double t_host0 = wall_ms();
    out = OpSet();
    out.side = O.side;
    out.cut = O.cut;
    out.state_class = O.state_class;
    out.state_layer = O.state_layer;
    std::vector<std::pair<int, int>> src;  // per new block: (class, O block)
    for (size_t c = 0; c < O.cls.size(); ++c) {
        OpClass nc;
        nc.dq = O.cls[c].dq;
        nc.states = O.cls[c].states;
        for (size_t bi = 0; bi < O.cls[c].blocks.size(); ++bi) {
            const OpBlock& ob = O.cls[c].blocks[bi];
            int qo = U.out.find(ob.Qo), qi = U.out.find(ob.Qi);
            if (qo < 0 || qi < 0 || U.off[qo] < 0 || U.off[qi] < 0) continue;
            nc.blocks.push_back({qo, qi, U.out.dim[qo], U.out.dim[qi], 0, ob.Qo, ob.Qi});
        }
        out.cls.push_back(std::move(nc));
    }
    alloc_env(C, out);
    // tmp[t] = O[t] U_Q2 : (T*dimQ) x k2, then new[t] = U_Q^T tmp[t]
    long long tmp_tot = 0;
    std::vector<long long> toff;
    for (size_t c = 0; c < out.cls.size(); ++c)
        for (const auto& nb : out.cls[c].blocks) {
            toff.push_back(tmp_tot);
            int bi = O.cls[c].find_block(U.basis.find(nb.Qi));
            (void)bi;
            tmp_tot += (long long)out.cls[c].states.size() * U.basis.dim[U.basis.find(nb.Qo)] * nb.cols;
        }
    // the intermediate is as large as the new environment times the enlarged
    // dimension over the kept one: from the block cache, given back on return
    C.scratch_tmp.ensure_cached(size_t(std::max<long long>(tmp_tot, 1)) * sizeof(double), C.cs);
    double* tmp = C.scratch_tmp.as<double>();
    // mixed form: both GEMM phases on the tensor cores in the sliced form when
    // the enlarged set's slices exist (FP64 GEMMs otherwise)
    double t_dev0 = wall_ms();
    C.timers[Ctx::T_REN_HOST] += t_dev0 - t_host0;
    if (C.cfg.precision == GBD_MIXED_BF16X3 && C.cfg.mixed_polish == 2 && tc_renormalize(C, O, U, out, toff, tmp)) {
        C.timers[Ctx::T_REN_TC_GFLOP] += renorm_flops(O, U, out) * 1e-9;
    } else {
        GBD_REQUIRE(O.resident(), GBD_ERR_STATE, "renormalisation: enlarged operators released and no sliced planes");
        const double t_plan0 = wall_ms();
        const double* dO = O.data.as<double>();
        const double* dU = U.data.as<double>();
        double* dN = out.data.as<double>();
        GemmPlan& PA = C.plan_a;
        GemmPlan& PB = C.plan_b;
        PA.clear();
        PB.clear();
        size_t j = 0;
        for (size_t c = 0; c < out.cls.size(); ++c) {
            int T = int(out.cls[c].states.size());
            for (const auto& nb : out.cls[c].blocks) {
                int eo = U.basis.find(nb.Qo), ei = U.basis.find(nb.Qi);
                int dimO = U.basis.dim[eo], dimI = U.basis.dim[ei];
                int bi = -1;
                for (size_t x = 0; x < O.cls[c].blocks.size(); ++x)
                    if (O.cls[c].blocks[x].qo == eo && O.cls[c].blocks[x].qi == ei) bi = int(x);
                GBD_REQUIRE(bi >= 0, GBD_ERR_STATE, "renormalisation: missing enlarged block");
                const OpBlock& ob = O.cls[c].blocks[bi];
                GemmTask ta{};
                ta.C = tmp + toff[j];
                ta.ldc = nb.cols;
                ta.M = T * dimO;
                ta.N = nb.cols;
                ta.nbatch = 1;
                GemmSeg ga{};
                ga.A = dO + ob.off;
                ga.lda = dimI;
                ga.B = dU + U.off[nb.qi];
                ga.ldb = nb.cols;
                ga.K = dimI;
                ga.T = 1;
                ga.coef = 1.0;
                PA.add_task(ta, {ga});
                GemmTask tb{};
                tb.C = dN + nb.off;
                tb.ldc = nb.cols;
                tb.M = nb.rows;
                tb.N = nb.cols;
                tb.nbatch = T;
                tb.bC = (long long)nb.rows * nb.cols;
                tb.bB = (long long)dimO * nb.cols;
                tb.bA = 0;
                GemmSeg gb{};
                gb.A = dU + U.off[nb.qo];
                gb.lda = nb.rows;
                gb.transA = 1;
                gb.B = tmp + toff[j];
                gb.ldb = nb.cols;
                gb.K = dimO;
                gb.T = 1;
                gb.coef = 1.0;
                PB.add_task(tb, {gb});
                ++j;
            }
        }
        std::vector<std::pair<const void*, size_t>> bufs = {{O.data.p, size_t(O.total) * 8},
                                                            {U.data.p, U.data.bytes},
                                                            {C.scratch_tmp.p, C.scratch_tmp.bytes},
                                                            {out.data.p, size_t(out.total) * 8}};
        PA.check(bufs, "renormalise/A");
        PB.check(bufs, "renormalise/B");
        C.timers[Ctx::T_REN_HOST] += wall_ms() - t_plan0;
        t_dev0 = wall_ms();
        C.timers[Ctx::T_REN_GFLOP] += (PA.flops + PB.flops) * 1e-9;
        PA.upload(C.cs);
        PA.launch(C.cs);
        PB.upload(C.cs);
        PB.launch(C.cs);
    }
    GBD_CHECK_CUDA(cudaStreamSynchronize(C.cs));
    C.scratch_tmp.release();
    C.timers[Ctx::T_REN_DEV] += wall_ms() - t_dev0;
}

// ============================================================== setup
void ensure_cuda(Ctx& C) {
    if (C.cuda_ready) return;
    GBD_CHECK_CUDA(cudaSetDevice(C.cfg.device));
    GBD_CHECK_CUDA(cudaStreamCreateWithFlags(&C.cs, cudaStreamNonBlocking));
    GBD_CHECK_CUDA(cudaStreamCreateWithFlags(&C.ios, cudaStreamNonBlocking));
    GBD_CHECK_CUDA(cudaEventCreate(&C.ev0));
    GBD_CHECK_CUDA(cudaEventCreate(&C.ev1));
    if (cusolverDnCreate(&C.sol) != CUSOLVER_STATUS_SUCCESS) throw Error(GBD_ERR_CUDA, "cusolverDnCreate failed");
    cusolverDnSetStream(C.sol, C.cs);
    if (cusolverDnCreateParams(&C.eig_params) != CUSOLVER_STATUS_SUCCESS)
        throw Error(GBD_ERR_CUDA, "cusolverDnCreateParams failed");
    for (int i = 0; i < Ctx::kEigStreams; ++i) {
        GBD_CHECK_CUDA(cudaStreamCreateWithFlags(&C.eig_st[i], cudaStreamNonBlocking));
        if (cusolverDnCreate(&C.eig_sol[i]) != CUSOLVER_STATUS_SUCCESS) throw Error(GBD_ERR_CUDA, "cusolverDnCreate failed");
        cusolverDnSetStream(C.eig_sol[i], C.eig_st[i]);
    }
    C.cuda_ready = true;
}

void destroy_ctx(Ctx& C) {
    if (!C.cuda_ready) return;
    cudaSetDevice(C.cfg.device);
    cudaDeviceSynchronize();
    auto free_host = [](HostEnv& h) {
        if (h.host) cudaFreeHost(h.host);
        if (h.meta) cudaFreeHost(h.meta);
        if (h.cks_host) cudaFreeHost(h.cks_host);
        if (h.cks_dev) cudaFree(h.cks_dev);
        if (h.done) cudaEventDestroy(h.done);
        if (h.loaded) cudaEventDestroy(h.loaded);
        h = HostEnv();
    };
    C.spill.reset();  // its IO thread finishes queued jobs before the buffers go
    for (auto& h : C.hostL) free_host(h);
    for (auto& h : C.hostR) free_host(h);
    C.pinned_bytes = 0;
    for (auto& ps : C.saves) { cudaEventDestroy(ps.a); cudaEventDestroy(ps.b); }
    C.saves.clear();
    C.hostL.clear();
    C.hostR.clear();
    if (C.sol) cusolverDnDestroy(C.sol);
    if (C.eig_params) cusolverDnDestroyParams(C.eig_params);
    C.eig_params = nullptr;
    for (int i = 0; i < Ctx::kEigStreams; ++i) {
        if (C.eig_sol[i]) cusolverDnDestroy(C.eig_sol[i]);
        if (C.eig_st[i]) cudaStreamDestroy(C.eig_st[i]);
        C.eig_work[i].release();
    }
    for (auto e : C.mark_pool) cudaEventDestroy(e);
    C.mark_pool.clear();
    C.marks.clear();
    if (C.ev0) cudaEventDestroy(C.ev0);
    if (C.ev1) cudaEventDestroy(C.ev1);
    C.envL.clear();
    C.envR.clear();
    // every holder of a cached block (stream-ordered on C.cs) gives it back
    // while C.cs still exists
    C.H = Heff();
    C.sites.clear();
    C.plan_a.free();
    C.plan_b.free();
    C.plan_c.free();
    cudaDeviceSynchronize();
    if (C.cs) cudaStreamDestroy(C.cs);
    if (C.ios) cudaStreamDestroy(C.ios);
    devcache_trim();
    C.cuda_ready = false;
}

void load_integrals(Ctx& C, int L, const double* h, const double* eri, double ecore) {
    GBD_REQUIRE(L >= 2 && L == C.cfg.L, GBD_ERR_ARG, "L must match the configuration and be >= 2");
    size_t n2 = size_t(L) * L, n4 = n2 * n2;
    double mx = 0.0;
    for (size_t i = 0; i < n2; ++i) mx = std::max(mx, std::fabs(h[i]));
    for (size_t i = 0; i < n4; ++i) mx = std::max(mx, std::fabs(eri[i]));
    double tol = 1e-12 * std::max(1.0, mx);
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j)
            GBD_REQUIRE(std::fabs(h[i * L + j] - h[j * L + i]) <= tol, GBD_ERR_ARG, "h is not symmetric");
    auto E = [&](int i, int j, int k, int l) { return eri[((size_t(i) * L + j) * L + k) * L + l]; };
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j)
            for (int k = 0; k < L; ++k)
                for (int l = 0; l < L; ++l) {
                    double v = E(i, j, k, l);
                    GBD_REQUIRE(std::fabs(v - E(j, i, k, l)) <= tol && std::fabs(v - E(k, l, i, j)) <= tol &&
                                    std::fabs(v - E(i, j, l, k)) <= tol,
                                GBD_ERR_ARG, "eri lacks the 8-fold symmetry");
                }
    C.L = L;
    C.h.assign(h, h + n2);
    C.eri.assign(eri, eri + n4);
    C.ecore = ecore;
    C.mpo.build(L, h, eri, C.cfg.switch_cut);
    for (auto& v : C.enl_links) v.clear();  // they follow the MPO
    C.have_ints = true;
    C.site_blocks_data.assign(L, {});
    C.site_blocks_meta.assign(L, {});
    C.site_kind.assign(L, -1);
    C.sites.clear();
    C.sites.resize(L);
    C.bonds.assign(L + 1, Bond());
    C.envL.clear();
    C.envR.clear();
    C.envL.resize(L + 1);
    C.envR.resize(L + 1);
    C.hostL.assign(L + 1, HostEnv());
    C.hostR.assign(L + 1, HostEnv());
    C.H = Heff();
    C.psi_valid = false;
}

void import_site(Ctx& C, int k, int kind, int nblk, const int* meta, const double* data) {
    GBD_REQUIRE(C.have_ints, GBD_ERR_STATE, "load integrals first");
    GBD_REQUIRE(k >= 0 && k < C.L && (kind == 0 || kind == 1) && nblk >= 0, GBD_ERR_ARG, "bad site arguments");
    long long tot = 0;
    for (int i = 0; i < nblk; ++i) {
        GBD_REQUIRE(meta[5 * i + 2] >= 0 && meta[5 * i + 2] < 4 && meta[5 * i + 3] >= 0 && meta[5 * i + 4] >= 0,
                    GBD_ERR_ARG, "bad block metadata");
        tot += (long long)meta[5 * i + 3] * meta[5 * i + 4];
    }
    C.site_blocks_meta[k].assign(meta, meta + 5 * nblk);
    C.site_blocks_data[k].assign(data, data + tot);
    C.site_kind[k] = kind;
}

// Site tensor k in the import format (Eq. 2 blocks): the imported blocks
// while the sites are not yet on the device, else the current isometry
// (after truncations) read back from the device.
void export_site(Ctx& C, int k, int* kind, std::vector<int>& meta, std::vector<double>& data) {
    GBD_REQUIRE(k >= 0 && k < C.L, GBD_ERR_ARG, "site out of range");
    GBD_REQUIRE(C.site_kind[k] >= 0, GBD_ERR_STATE, "site was never imported");
    const Iso& I = C.sites[k];
    meta.clear();
    data.clear();
    if (!I.data.p || I.kind < 0) {
        *kind = C.site_kind[k];
        meta = C.site_blocks_meta[k];
        data = C.site_blocks_data[k];
        return;
    }
    *kind = I.kind;
    std::vector<double> h(size_t(std::max<long long>(I.total, 1)));
    GBD_CHECK_CUDA(cudaStreamSynchronize(C.cs));
    if (I.total > 0) GBD_CHECK_CUDA(cudaMemcpy(h.data(), I.data.p, size_t(I.total) * sizeof(double), cudaMemcpyDeviceToHost));
    for (size_t oi = 0; oi < I.out.q.size(); ++oi) {
        if (I.off[oi] < 0) continue;
        const int e = I.basis.find(I.out.q[oi]);
        if (e < 0) continue;
        const int dout = I.out.dim[oi];
        for (const auto& sg : I.basis.segs[e]) {
            if (I.kind == 0) {  // rows: (left bond sector, s) segment; cols: new bond sector
                const Q ql{I.out.q[oi].n - kQS[sg.s].n, I.out.q[oi].t - kQS[sg.s].t};
                meta.insert(meta.end(), {ql.n, ql.t, sg.s, sg.size, dout});
                for (int i = 0; i < sg.size; ++i)
                    for (int j = 0; j < dout; ++j) data.push_back(h[I.off[oi] + (long long)(sg.off + i) * dout + j]);
            } else {            // rows: new bond sector; cols: (s, right bond sector) segment
                const Q ql = I.out.q[oi];
                meta.insert(meta.end(), {ql.n, ql.t, sg.s, dout, sg.size});
                for (int i = 0; i < dout; ++i)
                    for (int j = 0; j < sg.size; ++j) data.push_back(h[I.off[oi] + (long long)(sg.off + j) * dout + i]);
            }
        }
    }
}

// Bonds from imported blocks, then each site's isometry on the device.
static void make_iso(Ctx& C, int k, int kind) {
    Iso& I = C.sites[k];
    I = Iso();
    I.kind = kind;
    const auto& meta = C.site_blocks_meta[k];
    const auto& data = C.site_blocks_data[k];
    int nblk = int(meta.size() / 5);
    if (kind == 0) {
        I.basis = left_enlarged(C.bonds[k]);
        I.out = C.bonds[k + 1];
    } else {
        I.basis = right_enlarged(C.bonds[k + 1]);
        I.out = C.bonds[k];
    }
    I.off.assign(I.out.q.size(), -1);
    long long off = 0;
    for (size_t i = 0; i < I.out.q.size(); ++i) {
        int e = I.basis.find(I.out.q[i]);
        if (e < 0) continue;
        I.off[i] = off;
        off += (long long)I.basis.dim[e] * I.out.dim[i];
    }
    I.total = off;
    I.host.assign(size_t(std::max<long long>(off, 1)), 0.0);
    long long doff = 0;
    for (int b = 0; b < nblk; ++b) {
        Q ql{meta[5 * b], meta[5 * b + 1]};
        int s = meta[5 * b + 2], r = meta[5 * b + 3], c = meta[5 * b + 4];
        const double* blk = data.data() + doff;
        doff += (long long)r * c;
        if (r == 0 || c == 0) continue;
        if (kind == 0) {
            Q Qn = ql + kQS[s];
            int oi = I.out.find(Qn), e = I.basis.find(Qn);
            GBD_REQUIRE(oi >= 0 && e >= 0 && I.off[oi] >= 0, GBD_ERR_ARG, "site block outside the bonds");
            const Seg* sg = find_seg(I.basis, e, s);
            GBD_REQUIRE(sg && sg->size == r && I.out.dim[oi] == c, GBD_ERR_ARG, "site block dims disagree with bonds");
            for (int i = 0; i < r; ++i)
                for (int j = 0; j < c; ++j) I.host[I.off[oi] + (long long)(sg->off + i) * c + j] = blk[i * c + j];
        } else {
            int oi = I.out.find(ql), e = I.basis.find(ql);
            GBD_REQUIRE(oi >= 0 && e >= 0 && I.off[oi] >= 0, GBD_ERR_ARG, "site block outside the bonds");
            const Seg* sg = find_seg(I.basis, e, s);
            GBD_REQUIRE(sg && sg->size == c && I.out.dim[oi] == r, GBD_ERR_ARG, "site block dims disagree with bonds");
            for (int i = 0; i < r; ++i)
                for (int j = 0; j < c; ++j) I.host[I.off[oi] + (long long)(sg->off + j) * r + i] = blk[i * c + j];
        }
    }
    I.data.ensure(I.host.size() * sizeof(double));
    GBD_CHECK_CUDA(cudaMemcpyAsync(I.data.p, I.host.data(), I.host.size() * sizeof(double), cudaMemcpyHostToDevice, C.cs));
}

void finalize_sites(Ctx& C) {
    ensure_cuda(C);
    const int L = C.L;
    for (int k = 0; k < L; ++k) GBD_REQUIRE(C.site_kind[k] >= 0, GBD_ERR_STATE, "every site must be imported");
    std::vector<std::map<Q, int>> dims(L + 1);
    for (int k = 0; k < L; ++k) {
        const auto& meta = C.site_blocks_meta[k];
        for (size_t b = 0; b < meta.size() / 5; ++b) {
            Q ql{meta[5 * b], meta[5 * b + 1]};
            Q qr = ql + kQS[meta[5 * b + 2]];
            int r = meta[5 * b + 3], c = meta[5 * b + 4];
            auto chk = [&](std::map<Q, int>& m, const Q& q, int d) {
                auto it = m.find(q);
                if (it == m.end()) m[q] = d;
                else GBD_REQUIRE(it->second == d, GBD_ERR_ARG, "inconsistent bond dimension between sites");
            };
            chk(dims[k], ql, r);
            chk(dims[k + 1], qr, c);
        }
    }
    for (int k = 0; k <= L; ++k) {
        Bond b;
        for (auto& kv : dims[k])
            if (kv.second > 0) { b.q.push_back(kv.first); b.dim.push_back(kv.second); }
        C.bonds[k] = b;
    }
    GBD_REQUIRE(C.bonds[0].q.size() == 1 && C.bonds[0].q[0] == (Q{0, 0}), GBD_ERR_ARG, "bond 0 must be the vacuum");
    GBD_REQUIRE(C.bonds[L].q.size() == 1 && C.bonds[L].q[0] == (Q{C.cfg.N, C.cfg.tsz}), GBD_ERR_ARG,
                "bond L must carry (N, 2Sz)");
    for (int k = 0; k < L; ++k) make_iso(C, k, C.site_kind[k]);
    GBD_CHECK_CUDA(cudaStreamSynchronize(C.cs));
}

OpSet* env_of(Ctx& C, int side, int cut, bool create) {
    GBD_REQUIRE(cut >= 0 && cut <= C.L && (side == 0 || side == 1), GBD_ERR_ARG, "bad environment id");
    auto& v = side == 0 ? C.envL : C.envR;
    if (!v[cut] && create) v[cut] = std::make_unique<OpSet>();
    return v[cut].get();
}

void build_envs(Ctx& C, int b) {
    GBD_REQUIRE(b >= 0 && b + 1 < C.L, GBD_ERR_ARG, "two-site position out of range");
    finalize_sites(C);
    for (int k = 0; k < b; ++k) GBD_REQUIRE(C.site_kind[k] == 0, GBD_ERR_ARG, "sites left of b must be left-isometric");
    for (int k = b + 2; k < C.L; ++k)
        GBD_REQUIRE(C.site_kind[k] == 1, GBD_ERR_ARG, "sites right of b+1 must be right-isometric");
    // with offload on, every environment the position b does not use goes to
    // the pinned host store as soon as the next one is built from it, so the
    // device holds two or three environments at a time
    const bool off = C.cfg.offload != 0;
    C.envL[0] = trivial_env(C, 0);
    for (int k = 0; k < b; ++k) {
        OpSet O;
        EBasis eb;
        enlarge(C, *C.envL[k], 0, k, O, eb);
        auto E = std::make_unique<OpSet>();
        renormalize(C, O, C.sites[k], *E);
        C.envL[k + 1] = std::move(E);
        if (off) offload_env(C, 0, k);
    }
    C.envR[C.L] = trivial_env(C, 1);
    for (int k = C.L - 1; k >= b + 2; --k) {
        OpSet O;
        EBasis eb;
        enlarge(C, *C.envR[k + 1], 1, k, O, eb);
        auto E = std::make_unique<OpSet>();
        renormalize(C, O, C.sites[k], *E);
        C.envR[k] = std::move(E);
        if (off) offload_env(C, 1, k + 1);
    }
    C.H = Heff();
    C.psi_valid = false;
}

// Recomputation of an environment that was dropped without a host copy
// (env_recompute): from the nearest environment towards its chain end that
// is resident or stored, one enlargement + renormalisation per site with the
// current isometries (the steps of build_envs).  The environments passed on
// the way stay resident: the sweep needs them next.
void rebuild_env(Ctx& C, int side, int cut) {
    const double t0 = wall_ms();
    auto avail = [&](int c) {
        OpSet* E = env_of(C, side, c, false);
        if (!E) return false;
        const HostEnv& h = side == 0 ? C.hostL[c] : C.hostR[c];
        return E->resident() || h.valid;
    };
    int from = cut;
    if (side == 0) {
        while (from > 0 && !avail(from)) --from;
    } else {
        while (from < C.L && !avail(from)) ++from;
    }
    GBD_REQUIRE(avail(from), GBD_ERR_STATE, "no stored environment to recompute from");
    make_resident(C, side, from);
    int n = 0;
    if (side == 0) {
        for (int k = from; k < cut; ++k, ++n) {
            GBD_REQUIRE(C.sites[k].kind == 0, GBD_ERR_STATE, "recomputation needs left-isometric sites left of the cut");
            OpSet O;
            EBasis eb;
            enlarge(C, *C.envL[k], 0, k, O, eb);
            auto E = std::make_unique<OpSet>();
            renormalize(C, O, C.sites[k], *E);
            C.envL[k + 1] = std::move(E);
        }
    } else {
        for (int k = from - 1; k >= cut; --k, ++n) {
            GBD_REQUIRE(C.sites[k].kind == 1, GBD_ERR_STATE, "recomputation needs right-isometric sites right of the cut");
            OpSet O;
            EBasis eb;
            enlarge(C, *C.envR[k + 1], 1, k, O, eb);
            auto E = std::make_unique<OpSet>();
            renormalize(C, O, C.sites[k], *E);
            C.envR[k] = std::move(E);
        }
    }
    C.timers[Ctx::T_RECOMP_MS] += wall_ms() - t0;
    C.timers[Ctx::T_RECOMP_N] += n;
}

// ============================================================== H_eff
void setup_heff(Ctx& C, int b) {
    GBD_REQUIRE(b >= 0 && b + 1 < C.L, GBD_ERR_ARG, "two-site position out of range");
    OpSet* EL = C.envL[b].get();
    OpSet* ER = C.envR[b + 2].get();
    GBD_REQUIRE(EL && ER && EL->resident() && ER->resident(), GBD_ERR_STATE,
                "environments for this position are not built");
    Heff& H = C.H;
    H = Heff();
    H.b = b;
    enlarge(C, *EL, 0, b, H.OL, H.bL);
    enlarge(C, *ER, 1, b + 1, H.OR, H.bR);
    // wavefunction sectors: in both enlarged bases
    long long off = 0;
    for (size_t i = 0; i < H.bL.q.size(); ++i) {
        int j = H.bR.find(H.bL.q[i]);
        if (j < 0) continue;
        H.sq.push_back(H.bL.q[i]);
        H.sL.push_back(int(i));
        H.sR.push_back(j);
        H.soff.push_back(off);
        off += (long long)H.bL.dim[i] * H.bR.dim[j];
    }
    H.dim = off;
    GBD_REQUIRE(H.dim > 0, GBD_ERR_STATE, "empty wavefunction space");
    H.xin.ensure_cached(size_t(H.dim) * sizeof(double), C.cs);
    H.yout.ensure_cached(size_t(H.dim) * sizeof(double), C.cs);
    H.diag.ensure_cached(size_t(H.dim) * sizeof(double), C.cs);
    // phase 1: X_{c,Q2}[t] = OL[t][Q,Q2] psi[Q2]; phase 2: Y[Q] += sum X[t] OR[t][Q,Q2]^T
    long long xtot = 0;
    H.op_bytes = double(H.OL.total + H.OR.total) * 8.0;
    H.flops = 0.0;
    double nx = 0.0;
    for (size_t c = 0; c < H.OL.cls.size(); ++c) {
        const OpClass& cl = H.OL.cls[c];
        const OpClass& cr = H.OR.cls[c];
        GBD_REQUIRE(cl.dq == cr.dq && cl.states == cr.states, GBD_ERR_STATE, "class mismatch between enlarged blocks");
        int T = int(cl.states.size());
        for (size_t bi = 0; bi < cl.blocks.size(); ++bi) {
            const OpBlock& ob = cl.blocks[bi];
            int so = H.sector_of(ob.Qo), si = H.sector_of(ob.Qi);
            if (so < 0 || si < 0) continue;
            int br = -1;
            for (size_t x = 0; x < cr.blocks.size(); ++x)
                if (cr.blocks[x].Qo == ob.Qo && cr.blocks[x].Qi == ob.Qi) br = int(x);
            if (br < 0) continue;
            H.pairs.push_back({int(c), int(bi), br, so, si, xtot});
            const double mLo = H.bL.dim[H.sL[so]], mLi = H.bL.dim[H.sL[si]];
            const double mRo = H.bR.dim[H.sR[so]], mRi = H.bR.dim[H.sR[si]];
            xtot += (long long)T * H.bL.dim[H.sL[so]] * H.bR.dim[H.sR[si]];
            nx += double(T) * mLo * mRi;
            // useful flops: 2 M N K of both phases
            H.flops += 2.0 * T * mLo * mRi * mLi + 2.0 * mLo * mRo * (T * mRi);
            H.ngemm += 2LL * T;
        }
    }
    H.xtot = xtot;
    {
        // algorithmic bytes of one BF16x3 product: each operator element read
        // once (hi + lo), psi in and H psi out; the X round trip is overhead
        double elems = 0.0, padded = 0.0, xpad = 0.0;
        for (const OpSet* O : {&H.OL, &H.OR})
            for (const auto& c : O->cls)
                for (const auto& bb : c.blocks) {
                    elems += double(c.states.size()) * bb.rows * bb.cols;
                    padded += double(c.states.size()) * bb.rows * ((bb.cols + 7) / 8 * 8);
                }
        for (const auto& p : H.pairs)
            xpad += double(H.OL.cls[p.c].states.size()) * H.bL.dim[H.sL[p.s_out]] * ((H.bR.dim[H.sR[p.s_in]] + 7) / 8 * 8);
        H.mixed_bytes = 4.0 * elems + 16.0 * double(H.dim);
        H.mixed_x_bytes = 8.0 * nx;
        H.mem_ops = H.op_bytes;
        H.mem_bf16x3 = 4.0 * padded;
        H.mem_sliced = 8.0 * padded;
        H.mem_x64 = 8.0 * double(xtot);
        H.mem_xtc = 8.0 * xpad;
    }
    H.fp64_ready = false;
    H.diag_ready = false;
    H.tc_ready = false;
    GBD_CHECK_CUDA(cudaStreamSynchronize(C.cs));
}

// FP64 GEMM plans of the two phases, built at the first FP64 product of a
// position (mixed-precision runs may never need them).
void build_fp64_plans(Ctx& C) {
    Heff& H = C.H;
    H.X.ensure_cached(size_t(std::max<long long>(H.xtot, 1)) * sizeof(double), C.cs);
    const double* dOL = H.OL.data.as<double>();
    const double* dOR = H.OR.data.as<double>();
    double* dX = H.X.as<double>();
    double* din = H.xin.as<double>();
    double* dout = H.yout.as<double>();
    H.p1.clear();
    H.p2.clear();
    std::vector<std::vector<GemmSeg>> by_out(H.sq.size());
    for (const auto& p : H.pairs) {
        const OpClass& cl = H.OL.cls[p.c];
        const OpBlock& ob = cl.blocks[p.bl];
        const OpBlock& rb = H.OR.cls[p.c].blocks[p.br];
        int T = int(cl.states.size());
        int mLo = H.bL.dim[H.sL[p.s_out]], mLi = H.bL.dim[H.sL[p.s_in]];
        int mRo = H.bR.dim[H.sR[p.s_out]], mRi = H.bR.dim[H.sR[p.s_in]];
        GemmTask t1{};
        t1.C = dX + p.xoff;
        t1.ldc = mRi;
        t1.M = T * mLo;
        t1.N = mRi;
        t1.nbatch = 1;
        GemmSeg g1{};
        g1.A = dOL + ob.off;
        g1.lda = mLi;
        g1.B = din + H.soff[p.s_in];
        g1.ldb = mRi;
        g1.K = mLi;
        g1.T = 1;
        g1.coef = 1.0;
        H.p1.add_task(t1, {g1});
        GemmSeg g2{};
        g2.A = dX + p.xoff;
        g2.lda = mRi;
        g2.sA = (long long)mLo * mRi;
        g2.B = dOR + rb.off;
        g2.ldb = mRi;
        g2.sB = (long long)mRo * mRi;
        g2.transB = 1;
        g2.K = mRi;
        g2.T = T;
        g2.coef = 1.0;
        by_out[p.s_out].push_back(g2);
    }
    for (size_t s = 0; s < H.sq.size(); ++s) {
        GemmTask t2{};
        t2.C = dout + H.soff[s];
        t2.M = H.bL.dim[H.sL[s]];
        t2.N = H.bR.dim[H.sR[s]];
        t2.ldc = t2.N;
        t2.nbatch = 1;
        t2.beta = 0.0;
        H.p2.add_task(t2, by_out[s]);
    }
    std::vector<std::pair<const void*, size_t>> bufs = {{H.OL.data.p, size_t(H.OL.total) * 8},
                                                        {H.OR.data.p, size_t(H.OR.total) * 8},
                                                        {H.X.p, H.X.bytes}, {H.xin.p, H.xin.bytes},
                                                        {H.yout.p, H.yout.bytes}};
    H.p1.check(bufs, "heff/phase1");
    H.p2.check(bufs, "heff/phase2");
    H.p1.upload(C.cs);
    H.p2.upload(C.cs);
    GBD_CHECK_CUDA(cudaStreamSynchronize(C.cs));
    H.fp64_ready = true;
}


void apply_heff_dev(Ctx& C, const double* in, double* out, int precision) {
    // an FP64 product after the mixed form released the FP64 enlarged
    // operators (low-memory mode) enlarges them again
    const bool fp64 = precision == GBD_FP64 || precision == GBD_FP64_PER_BLOCK;
    if (fp64 && !(C.H.OL.resident() && C.H.OR.resident())) setup_heff(C, C.H.b);
    Heff& H = C.H;
    GBD_CHECK_CUDA(cudaMemcpyAsync(H.xin.p, in, size_t(H.dim) * sizeof(double), cudaMemcpyDeviceToDevice, C.cs));
    GBD_CHECK_CUDA(cudaEventRecord(C.ev0, C.cs));
    const bool two = precision == GBD_BF16X3_TWO_PHASE, fz = precision == GBD_BF16X3_FUSED;
    const bool tensor = precision == GBD_MIXED_BF16X3 || precision == GBD_SLICED_BF16 || two || fz;
    const int mode = precision == GBD_SLICED_BF16 ? 1 : 0;
    if (tensor) {
        // the BF16x3 plan is fused or two-phase: a request for the other form re-plans it
        const bool want_fused = fz || (precision == GBD_MIXED_BF16X3 && C.cfg.bf16x3_fused);
        if (mode == 0 && H.tc_ready && H.tc.pl[0].built && H.tc.pl[0].fused != want_fused) H.tc.pl[0].built = false;
        if (mode == 0) H.tc.want_fused = want_fused;
        if (!H.tc_ready || !H.tc.pl[mode].built) {
            const double tt0 = wall_ms();
            tc_prepare(C, mode);
            C.timers[Ctx::T_TCPREP] += wall_ms() - tt0;
            GBD_CHECK_CUDA(cudaEventRecord(C.ev0, C.cs));
        }
        tc_apply(C, mode);
    } else {
        if (!H.fp64_ready) {
            build_fp64_plans(C);
            GBD_CHECK_CUDA(cudaEventRecord(C.ev0, C.cs));
        }
        if (precision == GBD_FP64_PER_BLOCK) {
            H.p1.launch_per_task(C.cs);
            H.p2.launch_per_task(C.cs);
        } else {
            H.p1.launch(C.cs);
            H.p2.launch(C.cs);
        }
    }
    GBD_CHECK_CUDA(cudaEventRecord(C.ev1, C.cs));
    GBD_CHECK_CUDA(cudaMemcpyAsync(out, H.yout.p, size_t(H.dim) * sizeof(double), cudaMemcpyDeviceToDevice, C.cs));
    GBD_CHECK_CUDA(cudaEventSynchronize(C.ev1));
    if (tensor) {
        int e = tc_error(C);
        GBD_REQUIRE(e == 0, GBD_ERR_CUDA, "tensor-core product stopped on a bounded wait (code " + std::to_string(e) + ")");
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, C.ev0, C.ev1);
    C.ms_matvec_acc += ms;
    C.matvec_count += 1;
    if (precision == GBD_FP64_PER_BLOCK) {
        C.timers[Ctx::T_PROD_MS_PB] += ms;
        C.timers[Ctx::T_PROD_N_PB] += 1.0;
    } else if (two) {
        C.timers[Ctx::T_PROD_MS_TP] += ms;
        C.timers[Ctx::T_PROD_N_TP] += 1.0;
    } else if (fz) {
        C.timers[Ctx::T_PROD_MS_FZ] += ms;
        C.timers[Ctx::T_PROD_N_FZ] += 1.0;
    } else {
        C.timers[Ctx::T_PROD_MS0 + precision] += ms;
        C.timers[Ctx::T_PROD_N0 + precision] += 1.0;
        C.timers[Ctx::T_PROD_GF0 + precision] += H.flops * 1e-9;
    }
    if (precision == GBD_MIXED_BF16X3) {
        C.timers[Ctx::T_PROD_GB1] += H.mixed_bytes * 1e-9;
        if (!H.tc.pl[0].fused) C.timers[Ctx::T_PROD_XGB1] += H.mixed_x_bytes * 1e-9;  // the fused kernel keeps X on the SM
        tc_tune_step(C, ms);
    }
}

void heff_diag(Ctx& C) {
    if (!C.H.diag_ready && !(C.H.OL.resident() && C.H.OR.resident())) setup_heff(C, C.H.b);
    Heff& H = C.H;
    if (H.diag_ready) return;
    std::vector<DiagTask> tasks;
    std::vector<DiagSeg> segs;
    for (size_t s = 0; s < H.sq.size(); ++s) {
        DiagTask t{};
        t.out = H.diag.as<double>() + H.soff[s];
        t.mL = H.bL.dim[H.sL[s]];
        t.mR = H.bR.dim[H.sR[s]];
        t.seg0 = int(segs.size());
        for (size_t c = 0; c < H.OL.cls.size(); ++c) {
            const OpClass& cl = H.OL.cls[c];
            if (!(cl.dq == (Q{0, 0}))) continue;
            int bl = -1, br = -1;
            for (size_t x = 0; x < cl.blocks.size(); ++x)
                if (cl.blocks[x].Qo == H.sq[s] && cl.blocks[x].Qi == H.sq[s]) bl = int(x);
            const OpClass& cr = H.OR.cls[c];
            for (size_t x = 0; x < cr.blocks.size(); ++x)
                if (cr.blocks[x].Qo == H.sq[s] && cr.blocks[x].Qi == H.sq[s]) br = int(x);
            if (bl < 0 || br < 0) continue;
            segs.push_back({H.OL.data.as<double>() + cl.blocks[bl].off, H.OR.data.as<double>() + cr.blocks[br].off,
                            int(cl.states.size())});
        }
        t.nseg = int(segs.size()) - t.seg0;
        tasks.push_back(t);
    }
    heff_diagonal(tasks, segs, C.cs);
    GBD_CHECK_CUDA(cudaStreamSynchronize(C.cs));
    H.diag_ready = true;
}

// ============================================================== Davidson
namespace {
// cyclic Jacobi eigen-decomposition of a small symmetric matrix (n <= 64)
void jacobi(int n, std::vector<double> A, std::vector<double>& w, std::vector<double>& V) {
    V.assign(size_t(n) * n, 0.0);
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, nrm = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                nrm += A[i * n + j] * A[i * n + j];
                if (i != j) off += A[i * n + j] * A[i * n + j];
            }
        if (off <= 1e-32 * nrm || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return A[a * n + a] < A[b * n + b]; });
    w.resize(n);
    std::vector<double> Vs(size_t(n) * n);
    for (int j = 0; j < n; ++j) {
        w[j] = A[idx[j] * n + idx[j]];
        for (int i = 0; i < n; ++i) Vs[i * n + j] = V[i * n + idx[j]];
    }
    V.swap(Vs);
}
}  // namespace

int davidson(Ctx& C, double* psi_host, double* energy, gbd_dav_stats* st) {
    Heff& H = C.H;
    const long long n = H.dim;
    const int kmax = std::max(3, std::min(C.cfg.dav_max_sub, 36));
    const int keep = std::max(1, std::min(C.cfg.dav_keep, kmax - 2));
    const int prec = C.cfg.precision;
    // a BF16x3 product carries ~1e-5 relative rounding, so its residual cannot
    // fall much below that; the anchor products (below) fix the energy
    // (after the first anchor the subspace holds an exact pair and the
    // residual estimate follows the exact one down to dav_tol)
    double tol = prec == GBD_MIXED_BF16X3 ? std::max(C.cfg.dav_tol, 2e-5) : C.cfg.dav_tol;
    heff_diag(C);
    C.dav_V.ensure(size_t(kmax) * n * sizeof(double));
    C.dav_AV.ensure(size_t(kmax) * n * sizeof(double));
    C.dav_r.ensure(size_t(n) * sizeof(double));
    C.dav_t.ensure(size_t(n) * sizeof(double));
    C.dav_x.ensure(size_t(n) * sizeof(double));
    C.dav_ax.ensure(size_t(n) * sizeof(double));
    C.dav_tmp.ensure(size_t(keep) * n * sizeof(double));
    C.scratch_dot.ensure(multi_dot_partial_elems(40) * sizeof(double));
    C.scratch_small.ensure(128 * sizeof(double));
    double* V = C.dav_V.as<double>();
    double* AV = C.dav_AV.as<double>();
    double* r = C.dav_r.as<double>();
    double* t = C.dav_t.as<double>();
    double* x = C.dav_x.as<double>();
    double* ax = C.dav_ax.as<double>();
    double* part = C.scratch_dot.as<double>();
    double* small = C.scratch_small.as<double>();
    cudaStream_t s = C.cs;
    auto dots = [&](const double* Vb, int k, const double* y, std::vector<double>& out) {
        multi_dot(Vb, n, k, y, n, small, part, s);
        out.resize(k);
        GBD_CHECK_CUDA(cudaMemcpyAsync(out.data(), small, k * sizeof(double), cudaMemcpyDeviceToHost, s));
        GBD_CHECK_CUDA(cudaStreamSynchronize(s));
    };
    auto put = [&](const std::vector<double>& c) {
        GBD_CHECK_CUDA(cudaMemcpyAsync(small, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    };
    // start vector
    if (psi_host) {
        GBD_CHECK_CUDA(cudaMemcpyAsync(V, psi_host, size_t(n) * sizeof(double), cudaMemcpyHostToDevice, s));
    } else if (C.psi_valid && C.psi_b == H.b) {
        GBD_CHECK_CUDA(cudaMemcpyAsync(V, C.psi.p, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
        std::vector<double> v0(n);
        std::mt19937_64 rng(C.cfg.seed + 17 * H.b + 1);
        std::normal_distribution<double> nd;
        for (auto& v : v0) v = nd(rng);
        GBD_CHECK_CUDA(cudaMemcpyAsync(V, v0.data(), size_t(n) * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    std::vector<double> d;
    dots(V, 1, V, d);
    if (!(d[0] > 1e-28)) {
        std::vector<double> v0(n);
        std::mt19937_64 rng(C.cfg.seed + 31 * H.b + 7);
        std::normal_distribution<double> nd;
        for (auto& v : v0) v = nd(rng);
        GBD_CHECK_CUDA(cudaMemcpyAsync(V, v0.data(), size_t(n) * sizeof(double), cudaMemcpyHostToDevice, s));
        dots(V, 1, V, d);
    }
    scale(V, n, 1.0 / std::sqrt(d[0]), s);
    double ms_mv0 = C.ms_matvec_acc;
    // mixed form: the start vector's product is FP64, so the subspace holds
    // an exact pair from the first iteration (a converged start vector then
    // costs one FP64 product, as in the FP64 form)
    // used once the previous solve converged at its first anchor (late sweeps,
    // good start vectors); far from convergence it would only add an FP64 product
    const bool exact_start = prec == GBD_MIXED_BF16X3 && C.cfg.mixed_polish && C.last_dav_quick;
    // anchor products: FP64 GEMMs, or the sliced tensor-core form (~2^-30
    // relative to row maxima, well below the energy tolerance)
    const int anchor_prec = C.cfg.mixed_polish == 2 ? GBD_SLICED_BF16 : GBD_FP64;
    if (exact_start) {
        const double tp0 = wall_ms();
        apply_heff_dev(C, V, AV, anchor_prec);
        C.timers[Ctx::T_POLISH] += wall_ms() - tp0;
    } else {
        apply_heff_dev(C, V, AV, prec);
    }
    int nmv = 1, k = 1, iters = 0;
    // exact0: column 0 of AV is an accurate product (the exact start, or the
    // anchored pair after a restart).  H is symmetric, so the projections of
    // later columns onto it are taken on its accurate side, (H x) . v,
    // instead of x . (H v) with v's mixed product: only the block of the
    // correction directions then carries the mixed products' rounding, and
    // each anchor round shrinks the exact residual instead of converging
    // back to the mixed operator's eigenvector.  A full subspace then
    // restarts through an anchor (not a thick restart, whose kept vectors
    // would mix accurate and mixed products).
    bool exact0 = exact_start;
    std::vector<double> Hs(size_t(kmax) * kmax, 0.0);
    dots(V, 1, AV, d);
    Hs[0] = d[0];
    double theta = 0.0, rn = 0.0;
    std::vector<double> w, S;
    std::vector<double> hist;  // residual norms, for the mixed-precision stagnation test
    int anchors = 0;
    double anchor_rn[GBD_MAX_ANCHORS] = {0.0};
    // the anchored pair with the smallest exact residual (a later anchor can
    // come out worse once the mixed products' rounding floor is reached)
    double best_rn = -1.0, best_theta = 0.0;
    int status = GBD_OK;
    while (true) {
        ++iters;
        std::vector<double> A(size_t(k) * k);
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) A[i * k + j] = 0.5 * (Hs[i * kmax + j] + Hs[j * kmax + i]);
        jacobi(k, A, w, S);
        theta = w[0];
        std::vector<double> s0(k);
        for (int i = 0; i < k; ++i) s0[i] = S[i * k + 0];
        put(s0);
        combine(V, n, k, small, x, n, 1.0, 0.0, s);
        combine(AV, n, k, small, ax, n, 1.0, 0.0, s);
        axpby(ax, r, n, 1.0, 0.0, s);
        axpby(x, r, n, -theta, 1.0, s);
        dots(r, 1, r, d);
        rn = std::sqrt(std::max(0.0, d[0]));
        bool anchor = false;
        if (prec == GBD_MIXED_BF16X3 && C.cfg.mixed_polish) {
            // Mixed products carry ~1e-5 relative noise, so the residual stalls
            // at a floor that grows with |theta|.  At the floor (or at the
            // tolerance) the Ritz vector is anchored: one accurate product
            // (sliced or FP64) gives its exact residual; if that is below the
            // tolerance we are done, otherwise the subspace restarts from the
            // exact pair and further mixed directions only correct it (exact0
            // below), which shrinks the exact residual round by round.
            hist.push_back(rn);
            bool stalled = false;
            if (hist.size() > 9) {
                const size_t n8 = hist.size() - 6;
                double before = *std::min_element(hist.begin(), hist.begin() + n8);
                double recent = *std::min_element(hist.begin() + n8, hist.end());
                // < 10% gain in 6 iterations, near the mixed floor (~1e-5 |theta|)
                stalled = recent > 0.9 * before && rn <= 1e-4 * std::max(1.0, std::fabs(theta));
            }
            // before the first anchor the mixed residual cannot go much below
            // the products' rounding (~3e-6 |theta| measured): anchor at
            // 1e-5 |theta| rather than iterate at the floor
            const double first = anchors == 0 ? 1e-5 * std::fabs(theta) : 0.0;
            anchor = rn <= std::max(tol, first) || stalled || nmv >= C.cfg.dav_max_matvec || (exact0 && k >= kmax);
            if (k == 1 && exact_start && anchors == 0 && iters == 1) {
                // the residual of the start vector is already exact
                if (rn <= C.cfg.dav_tol) break;
                anchor = false;
            }
        } else if (rn <= tol) {
            break;
        }
        if (anchor) {
            const double tp0 = wall_ms();
            apply_heff_dev(C, x, ax, anchor_prec);
            C.timers[Ctx::T_POLISH] += wall_ms() - tp0;
            ++nmv;
            ++anchors;
            dots(x, 1, x, d);
            const double xn = std::sqrt(d[0]);
            scale(x, n, 1.0 / xn, s);
            scale(ax, n, 1.0 / xn, s);
            dots(x, 1, ax, d);
            theta = d[0];
            axpby(ax, r, n, 1.0, 0.0, s);
            axpby(x, r, n, -theta, 1.0, s);
            dots(r, 1, r, d);
            rn = std::sqrt(std::max(0.0, d[0]));
            anchor_rn[std::min(anchors, GBD_MAX_ANCHORS) - 1] = rn;
            if (rn <= C.cfg.dav_tol) break;
            const double prev_best = best_rn;
            if (best_rn < 0.0 || rn < best_rn) {
                C.dav_best.ensure(size_t(n) * sizeof(double));
                GBD_CHECK_CUDA(cudaMemcpyAsync(C.dav_best.p, x, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, s));
                best_rn = rn;
                best_theta = theta;
            }
            // the mixed products' rounding floor: an anchor round that does not
            // cut the best exact residual by a fifth, or the last allowed
            // anchor (far from convergence, with a small gap, rounds are
            // slower but still gain; at the floor they gain nothing)
            if (anchors >= GBD_MAX_ANCHORS || (prev_best >= 0.0 && rn > 0.8 * prev_best)) {
                status = GBD_WARN_PRECISION_FLOOR;
                break;
            }
            tol = C.cfg.dav_tol;
            if (nmv >= C.cfg.dav_max_matvec) { status = GBD_WARN_NOT_CONVERGED; break; }
            // restart from the exact pair (x, H x)
            GBD_CHECK_CUDA(cudaMemcpyAsync(V, x, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, s));
            GBD_CHECK_CUDA(cudaMemcpyAsync(AV, ax, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, s));
            std::fill(Hs.begin(), Hs.end(), 0.0);
            Hs[0] = theta;
            k = 1;
            exact0 = true;
            hist.clear();
        }
        if (nmv >= C.cfg.dav_max_matvec) { status = GBD_WARN_NOT_CONVERGED; break; }
        precondition(r, H.diag.as<double>(), theta, t, n, s);
        // two Gram-Schmidt passes on the device: the projections stay in
        // `small` (no host round trip), t -= sum_i (V_i . t) V_i
        auto orth = [&](int kk) {
            for (int pass = 0; pass < 2; ++pass) {
                multi_dot(V, n, kk, t, n, small, part, s);
                combine(V, n, kk, small, t, n, -1.0, 1.0, s);
            }
        };
        orth(k);
        dots(t, 1, t, d);
        double tn = std::sqrt(std::max(0.0, d[0]));
        if (tn < 1e-10 * std::max(rn, 1e-300)) {  // fall back to the plain residual
            axpby(r, t, n, 1.0, 0.0, s);
            orth(k);
            dots(t, 1, t, d);
            tn = std::sqrt(std::max(0.0, d[0]));
            if (tn < 1e-300) break;
        }
        scale(t, n, 1.0 / tn, s);
        if (k >= kmax) {  // thick restart with the lowest `keep` Ritz vectors
            double* tmp = C.dav_tmp.as<double>();
            for (int j = 0; j < keep; ++j) {
                std::vector<double> cj(k);
                for (int i = 0; i < k; ++i) cj[i] = S[i * k + j];
                put(cj);
                combine(V, n, k, small, tmp + size_t(j) * n, n, 1.0, 0.0, s);
            }
            GBD_CHECK_CUDA(cudaMemcpyAsync(V, tmp, size_t(keep) * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            for (int j = 0; j < keep; ++j) {
                std::vector<double> cj(k);
                for (int i = 0; i < k; ++i) cj[i] = S[i * k + j];
                put(cj);
                combine(AV, n, k, small, tmp + size_t(j) * n, n, 1.0, 0.0, s);
            }
            GBD_CHECK_CUDA(cudaMemcpyAsync(AV, tmp, size_t(keep) * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            std::fill(Hs.begin(), Hs.end(), 0.0);
            for (int j = 0; j < keep; ++j) Hs[j * kmax + j] = w[j];
            k = keep;
            exact0 = false;
            orth(k);
            dots(t, 1, t, d);
            scale(t, n, 1.0 / std::sqrt(std::max(d[0], 1e-300)), s);
        }
        GBD_CHECK_CUDA(cudaMemcpyAsync(V + size_t(k) * n, t, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, s));
        apply_heff_dev(C, V + size_t(k) * n, AV + size_t(k) * n, prec);
        ++nmv;
        std::vector<double> hcol;
        if (exact0 && prec == GBD_MIXED_BF16X3) {
            // V^T (H v) and (H x) . v on the accurate side, one host round trip
            multi_dot(V, n, k + 1, AV + size_t(k) * n, n, small, part, s);
            multi_dot(AV, n, 1, V + size_t(k) * n, n, small + k + 1, part, s);
            hcol.resize(k + 2);
            GBD_CHECK_CUDA(cudaMemcpyAsync(hcol.data(), small, (k + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
            GBD_CHECK_CUDA(cudaStreamSynchronize(s));
            hcol[0] = hcol[k + 1];
        } else {
            dots(V, k + 1, AV + size_t(k) * n, hcol);
        }
        for (int i = 0; i <= k; ++i) {
            Hs[i * kmax + k] = hcol[i];
            Hs[k * kmax + i] = hcol[i];
        }
        ++k;
    }
    // a mixed Davidson that stopped on a warning returns its best anchored
    // pair (exact Rayleigh quotient, smallest exact residual) unless the
    // current pair is an anchored one at least as good
    if (prec == GBD_MIXED_BF16X3 && status != GBD_OK && best_rn >= 0.0) {
        const bool cur_anchored = anchors > 0 && anchor_rn[std::min(anchors, GBD_MAX_ANCHORS) - 1] == rn;
        if (!cur_anchored || best_rn < rn) {
            GBD_CHECK_CUDA(cudaMemcpyAsync(x, C.dav_best.p, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, s));
            rn = best_rn;
            theta = best_theta;
        }
    }
    // normalised Ritz vector becomes the current two-site vector
    dots(x, 1, x, d);
    scale(x, n, 1.0 / std::sqrt(d[0]), s);
    if (prec == GBD_MIXED_BF16X3) C.last_dav_quick = (rn <= C.cfg.dav_tol) && anchors <= 1 && status == GBD_OK;
    C.psi.ensure(size_t(n) * sizeof(double));
    GBD_CHECK_CUDA(cudaMemcpyAsync(C.psi.p, x, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (psi_host) GBD_CHECK_CUDA(cudaMemcpyAsync(psi_host, x, size_t(n) * sizeof(double), cudaMemcpyDeviceToHost, s));
    GBD_CHECK_CUDA(cudaStreamSynchronize(s));
    C.psi_valid = true;
    C.psi_b = H.b;
    if (energy) *energy = theta + C.ecore;
    if (st) {
        st->energy = theta + C.ecore;
        st->resid = rn;
        st->matvecs = nmv;
        st->iterations = iters;
        st->ms_matvec = C.ms_matvec_acc - ms_mv0;
        st->anchors = anchors;
        for (int i = 0; i < GBD_MAX_ANCHORS; ++i) st->anchor_resid[i] = anchor_rn[i];
    }
    return status;
}

// ============================================================== truncation
namespace {
__global__ void gather_eigvec_kernel(const double* __restrict__ A, int lda, int m, int k, double* __restrict__ U) {
    // U[i][a] = row i < m of eigenvector (lda-1-a) (ascending order from the
    // eigensolver, column-major A of an lda x lda slot)
    long long n = (long long)m * k;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        int i = int(e / k), a = int(e % k);
        U[e] = A[(long long)(lda - 1 - a) * lda + i];
    }
}

struct Pick {
    double lam;
    int sec, idx;
};
}  // namespace

// Post-processing of Sec. II.B step 3 on the current two-site vector.
// dir = +1: keep states of the enlarged left block, new left-isometric site b,
// new left environment at cut b+1, start vector at b+1.  dir = -1: the
// mirror image on the right, start vector at b-1.
double truncate_step(Ctx& C, int dir, int Dmax) {
    Heff& H = C.H;
    const int b = H.b;
    GBD_REQUIRE(C.psi_valid && C.psi_b == b, GBD_ERR_STATE, "no two-site vector at this position");
    GBD_REQUIRE(dir == 1 || dir == -1, GBD_ERR_ARG, "dir must be +1 or -1");
    GBD_REQUIRE(Dmax >= 1, GBD_ERR_ARG, "Dmax must be >= 1");
    if (dir == 1) GBD_REQUIRE(b + 2 < C.L, GBD_ERR_ARG, "no site to the right");
    if (dir == -1) GBD_REQUIRE(b >= 1, GBD_ERR_ARG, "no site to the left");
    cudaStream_t s = C.cs;
    const double* psi = C.psi.as<double>();
    const int ns = int(H.sq.size());
    // density matrices, grouped in size classes: sector i's m_i x m_i block
    // sits in the top-left corner of an npad x npad slot of its class (npad =
    // m rounded up to 16, then to 32), the rest of the slot is -I, which
    // leaves rho's eigenpairs untouched (block diagonal) and sorts its own
    // eigenvalues (-1) below rho's (>= 0)
    std::vector<int> m(ns), npad(ns), cls_of(ns), slot(ns);
    std::vector<long long> roff(ns), eoff(ns);
    std::map<int, std::vector<int>> by_pad;  // npad -> sectors
    for (int i = 0; i < ns; ++i) {
        m[i] = dir == 1 ? H.bL.dim[H.sL[i]] : H.bR.dim[H.sR[i]];
        npad[i] = m[i] <= 16 ? 16 : (m[i] + 31) / 32 * 32;
        if (m[i] > 0) by_pad[npad[i]].push_back(i);
    }
    struct EigClass { int n, batch; long long a0, w0; int i0; };  // i0: first info entry
    std::vector<EigClass> ecls;
    long long rtot = 0, etot = 0;
    int ninfo = 0;
    for (auto& kv : by_pad) {
        EigClass ec{kv.first, int(kv.second.size()), rtot, etot, ninfo};
        ninfo += ec.batch;
        for (size_t j = 0; j < kv.second.size(); ++j) {
            const int i = kv.second[j];
            cls_of[i] = int(ecls.size());
            slot[i] = int(j);
            roff[i] = rtot + (long long)j * ec.n * ec.n;
            eoff[i] = etot + (long long)j * ec.n;
        }
        rtot += (long long)ec.batch * ec.n * ec.n;
        etot += (long long)ec.batch * ec.n;
        ecls.push_back(ec);
    }
    DevBuf rho, evals, info;
    rho.ensure_cached(size_t(std::max<long long>(rtot, 1)) * sizeof(double), s);
    evals.ensure_cached(size_t(std::max<long long>(etot, 1)) * sizeof(double), s);
    info.ensure_cached(sizeof(int) * (ninfo + 1), s);
    if (!C.marks.empty()) step_mark(C, Ctx::T_PH_RHO_EIG);
    if (rtot > 0) {
        GBD_CHECK_CUDA(cudaMemsetAsync(rho.p, 0, size_t(rtot) * sizeof(double), s));
        std::vector<PadSeg> pads;
        for (int i = 0; i < ns; ++i)
            if (m[i] > 0 && npad[i] > m[i]) pads.push_back({rho.as<double>() + roff[i], npad[i], m[i]});
        pad_identity(pads, -1.0, s);
    }
    GemmPlan& P = C.plan_c;
    P.clear();
    for (int i = 0; i < ns; ++i) {
        if (m[i] == 0) continue;
        int mL = H.bL.dim[H.sL[i]], mR = H.bR.dim[H.sR[i]];
        GemmTask t{};
        t.C = rho.as<double>() + roff[i];
        t.ldc = npad[i];
        t.M = m[i];
        t.N = m[i];
        t.nbatch = 1;
        GemmSeg g{};
        g.A = psi + H.soff[i];
        g.B = psi + H.soff[i];
        g.T = 1;
        g.coef = 1.0;
        if (dir == 1) { g.lda = mR; g.ldb = mR; g.transB = 1; g.K = mR; }
        else { g.lda = mR; g.ldb = mR; g.transA = 1; g.K = mL; }
        P.add_task(t, {g});
    }
    P.check({{C.psi.p, C.psi.bytes}, {rho.p, rho.bytes}}, "truncate/rho");
    P.upload(s);
    P.launch(s);
    // eigen-decomposition (FP64, cuSOLVER): one batched solve per size class,
    // the classes spread over several streams (largest first) so they overlap
    const double t_eig0 = wall_ms();
    cudaEvent_t e_rho;
    GBD_CHECK_CUDA(cudaEventCreateWithFlags(&e_rho, cudaEventDisableTiming));
    GBD_CHECK_CUDA(cudaEventRecord(e_rho, s));
    std::vector<int> corder(ecls.size());
    std::iota(corder.begin(), corder.end(), 0);
    std::sort(corder.begin(), corder.end(), [&](int a, int b) { return ecls[a].n > ecls[b].n; });
    size_t wd_need[Ctx::kEigStreams] = {0}, wh_need[Ctx::kEigStreams] = {0};
    std::vector<size_t> wd_of(ecls.size()), wh_of(ecls.size());
    for (size_t j = 0; j < corder.size(); ++j) {
        const EigClass& ec = ecls[corder[j]];
        const int k = int(j % Ctx::kEigStreams);
        size_t wd = 0, wh = 0;
        if (cusolverDnXsyevBatched_bufferSize(C.eig_sol[k], C.eig_params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                              ec.n, CUDA_R_64F, rho.as<double>() + ec.a0, ec.n, CUDA_R_64F,
                                              evals.as<double>() + ec.w0, CUDA_R_64F, &wd, &wh,
                                              ec.batch) != CUSOLVER_STATUS_SUCCESS)
            throw Error(GBD_ERR_CUDA, "batched syev buffer size query failed");
        wd_need[k] = std::max(wd_need[k], wd);
        wh_need[k] = std::max(wh_need[k], wh);
    }
    for (int k = 0; k < Ctx::kEigStreams; ++k) {
        if (wd_need[k] > C.eig_work[k].bytes) C.eig_work[k].ensure(std::max<size_t>(wd_need[k], 16));
        if (wh_need[k] > C.eig_host[k].size()) C.eig_host[k].resize(wh_need[k]);
        GBD_CHECK_CUDA(cudaStreamWaitEvent(C.eig_st[k], e_rho, 0));
    }
    for (size_t j = 0; j < corder.size(); ++j) {
        const EigClass& ec = ecls[corder[j]];
        const int k = int(j % Ctx::kEigStreams);
        if (cusolverDnXsyevBatched(C.eig_sol[k], C.eig_params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, ec.n,
                                   CUDA_R_64F, rho.as<double>() + ec.a0, ec.n, CUDA_R_64F, evals.as<double>() + ec.w0,
                                   CUDA_R_64F, C.eig_work[k].p, C.eig_work[k].bytes,
                                   C.eig_host[k].empty() ? nullptr : C.eig_host[k].data(), C.eig_host[k].size(),
                                   info.as<int>() + ec.i0, ec.batch) != CUSOLVER_STATUS_SUCCESS)
            throw Error(GBD_ERR_CUDA, "batched syev failed");
    }
    for (int k = 0; k < Ctx::kEigStreams; ++k) {
        cudaEvent_t e;
        GBD_CHECK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        GBD_CHECK_CUDA(cudaEventRecord(e, C.eig_st[k]));
        GBD_CHECK_CUDA(cudaStreamWaitEvent(s, e, 0));
        cudaEventDestroy(e);
    }
    cudaEventDestroy(e_rho);
    std::vector<double> ev(size_t(std::max<long long>(etot, 1)));
    std::vector<int> hinfo(ninfo + 1);
    if (etot > 0)
        GBD_CHECK_CUDA(cudaMemcpyAsync(ev.data(), evals.p, size_t(etot) * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (ninfo > 0)
        GBD_CHECK_CUDA(cudaMemcpyAsync(hinfo.data(), info.p, ninfo * sizeof(int), cudaMemcpyDeviceToHost, s));
    GBD_CHECK_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < ninfo; ++c) GBD_REQUIRE(hinfo[c] == 0, GBD_ERR_CUDA, "eigensolver did not converge");
    // rho's eigenvalues are the last m_i of its slot's npad_i (ascending)
    for (int i = 0; i < ns; ++i) eoff[i] += npad[i] - m[i];
    C.timers[Ctx::T_EIG] += wall_ms() - t_eig0;
    // global selection: descending, at most Dmax, degenerate group at the cut
    // moves the cut down, sqrt(lambda) <= 1e-13 sqrt(lambda_max) dropped
    std::vector<Pick> all;
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j < m[i]; ++j) all.push_back({std::max(0.0, ev[eoff[i] + m[i] - 1 - j]), i, j});
    std::stable_sort(all.begin(), all.end(), [](const Pick& a, const Pick& b) {
        if (a.lam != b.lam) return a.lam > b.lam;
        if (a.sec != b.sec) return a.sec < b.sec;
        return a.idx < b.idx;
    });
    int nall = int(all.size());
    int keep = std::min(Dmax, nall);
    auto sig = [&](int i) { return std::sqrt(all[i].lam); };
    if (keep < nall && keep > 0) {
        double ref = sig(keep - 1);
        double tolr = 1e-10 * std::max(ref, 1e-300);
        if (std::fabs(sig(keep) - ref) <= tolr) {
            int j = keep - 1;
            while (j > 0 && std::fabs(sig(j - 1) - ref) <= tolr) --j;
            keep = std::max(j, 1);
        }
    }
    double smax = nall ? sig(0) : 0.0;
    while (keep > 1 && sig(keep - 1) <= 1e-13 * smax) --keep;
    std::vector<int> kept(ns, 0);
    double kept_sum = 0.0;
    for (int i = 0; i < keep; ++i) { kept[all[i].sec]++; kept_sum += all[i].lam; }
    double weight = std::max(0.0, 1.0 - kept_sum);
    // new bond and isometry
    Bond nb;
    for (int i = 0; i < ns; ++i)
        if (kept[i] > 0) { nb.q.push_back(H.sq[i]); nb.dim.push_back(kept[i]); }
    Iso I;
    I.kind = dir == 1 ? 0 : 1;
    I.basis = dir == 1 ? H.bL : H.bR;
    I.out = nb;
    I.off.assign(nb.q.size(), -1);
    long long itot = 0;
    for (size_t i = 0; i < nb.q.size(); ++i) {
        I.off[i] = itot;
        itot += (long long)I.basis.dim[I.basis.find(nb.q[i])] * nb.dim[i];
    }
    I.total = itot;
    I.data.ensure_cached(size_t(std::max<long long>(itot, 1)) * sizeof(double), s);
    // C = U^T psi (dir +1) or psi V (dir -1), per kept sector
    std::vector<long long> coff(nb.q.size());
    long long ctot = 0;
    for (size_t i = 0; i < nb.q.size(); ++i) {
        int si = H.sector_of(nb.q[i]);
        int other = dir == 1 ? H.bR.dim[H.sR[si]] : H.bL.dim[H.sL[si]];
        coff[i] = ctot;
        ctot += (long long)nb.dim[i] * other;
    }
    DevBuf Cbuf;
    Cbuf.ensure_cached(size_t(std::max<long long>(ctot, 1)) * sizeof(double), s);
    P.clear();
    for (size_t i = 0; i < nb.q.size(); ++i) {
        int si = H.sector_of(nb.q[i]);
        int k = nb.dim[i];
        long long nel = (long long)m[si] * k;
        gather_eigvec_kernel<<<unsigned(std::min<long long>((nel + 255) / 256, 4096)), 256, 0, s>>>(
            rho.as<double>() + roff[si], npad[si], m[si], k, I.data.as<double>() + I.off[i]);
        count_launch();
        int mL = H.bL.dim[H.sL[si]], mR = H.bR.dim[H.sR[si]];
        GemmTask t{};
        t.C = Cbuf.as<double>() + coff[i];
        t.nbatch = 1;
        GemmSeg g{};
        g.T = 1;
        g.coef = 1.0;
        if (dir == 1) {  // (k x mL) (mL x mR)
            t.M = k; t.N = mR; t.ldc = mR;
            g.A = I.data.as<double>() + I.off[i]; g.lda = k; g.transA = 1;
            g.B = psi + H.soff[si]; g.ldb = mR; g.K = mL;
        } else {         // (mL x mR) (mR x k)
            t.M = mL; t.N = k; t.ldc = k;
            g.A = psi + H.soff[si]; g.lda = mR;
            g.B = I.data.as<double>() + I.off[i]; g.ldb = k; g.K = mR;
        }
        P.add_task(t, {g});
    }
    GBD_CHECK_CUDA(cudaGetLastError());
    P.check({{C.psi.p, C.psi.bytes}, {I.data.p, I.data.bytes}, {Cbuf.p, Cbuf.bytes}}, "truncate/C");
    P.upload(s);
    P.launch(s);
    // the position's products are done: only the sliced operator planes (read
    // by the renormalisation) stay on the device
    if (H.tc_ready) tc_release_products(C);
    // renormalised environment of the truncated block (Sec. II.B step 3)
    auto E = std::make_unique<OpSet>();
    if (!C.marks.empty()) step_mark(C, Ctx::T_PH_RENORM);
    if (dir == 1) renormalize(C, H.OL, I, *E);
    else renormalize(C, H.OR, I, *E);
    if (!C.marks.empty()) step_mark(C, Ctx::T_PH_NEXT);
    // next two-site vector ("StVec")
    const int L = C.L;
    if (dir == 1) {
        C.bonds[b + 1] = nb;
        const Iso& Bn = C.sites[b + 2];
        GBD_REQUIRE(Bn.kind == 1, GBD_ERR_STATE, "site b+2 must be right-isometric");
        EBasis nL = left_enlarged(C.bonds[b + 1]);
        EBasis nR = right_enlarged(C.bonds[b + 3]);
        std::vector<Q> sq;
        std::vector<long long> so;
        std::vector<int> sLi, sRi;
        long long off = 0;
        for (size_t i = 0; i < nL.q.size(); ++i) {
            int j = nR.find(nL.q[i]);
            if (j < 0) continue;
            sq.push_back(nL.q[i]); sLi.push_back(int(i)); sRi.push_back(j); so.push_back(off);
            off += (long long)nL.dim[i] * nR.dim[j];
        }
        C.psi.ensure(size_t(std::max<long long>(off, 1)) * sizeof(double));
        GBD_CHECK_CUDA(cudaMemsetAsync(C.psi.p, 0, size_t(std::max<long long>(off, 1)) * sizeof(double), s));
        P.clear();
        for (size_t i = 0; i < nb.q.size(); ++i) {  // q = new bond b+1 sector
            int si = H.sector_of(nb.q[i]);
            int eR = H.sR[si];
            for (const auto& sg2 : H.bR.segs[eR]) {   // s2, qn = q + q_s2 at cut b+2
                Q qn = C.bonds[b + 2].q[sg2.bq];
                Q Qp = nb.q[i] + kQS[sg2.s];          // new enlarged-left sector
                auto it = std::lower_bound(sq.begin(), sq.end(), Qp);
                if (it == sq.end() || *it != Qp) continue;
                int ps = int(it - sq.begin());
                const Seg* sl = find_seg(nL, sLi[ps], sg2.s);
                int vo = Bn.out.find(qn);
                int ve = Bn.basis.find(qn);
                if (!sl || vo < 0 || ve < 0 || Bn.off[vo] < 0) continue;
                for (const auto& sg3 : Bn.basis.segs[ve]) {  // s3, cut-(b+3) sector
                    const Seg* sr = find_seg(nR, sRi[ps], sg3.s);
                    if (!sr) continue;
                    GemmTask t{};
                    int ldn = nR.dim[sRi[ps]];
                    t.C = C.psi.as<double>() + so[ps] + (long long)sl->off * ldn + sr->off;
                    t.ldc = ldn;
                    t.M = nb.dim[i];
                    t.N = sg3.size;
                    t.nbatch = 1;
                    t.beta = 0.0;
                    GemmSeg g{};
                    g.A = Cbuf.as<double>() + coff[i] + sg2.off;
                    g.lda = H.bR.dim[eR];
                    g.B = Bn.data.as<double>() + Bn.off[vo] + (long long)sg3.off * Bn.out.dim[vo];
                    g.ldb = Bn.out.dim[vo];
                    g.transB = 1;
                    g.K = sg2.size;
                    g.T = 1;
                    g.coef = 1.0;
                    P.add_task(t, {g});
                }
            }
        }
        P.check({{C.psi.p, C.psi.bytes}, {Cbuf.p, Cbuf.bytes}, {Bn.data.p, Bn.data.bytes}}, "truncate/next+");
        P.upload(s);
        P.launch(s);
        C.psi_b = b + 1;
        C.sites[b] = std::move(I);
        C.site_kind[b] = 0;
        C.envL[b + 1] = std::move(E);
    } else {
        C.bonds[b + 1] = nb;
        const Iso& Ap = C.sites[b - 1];
        GBD_REQUIRE(Ap.kind == 0, GBD_ERR_STATE, "site b-1 must be left-isometric");
        EBasis nL = left_enlarged(C.bonds[b - 1]);
        EBasis nR = right_enlarged(C.bonds[b + 1]);
        std::vector<Q> sq;
        std::vector<long long> so;
        std::vector<int> sLi, sRi;
        long long off = 0;
        for (size_t i = 0; i < nL.q.size(); ++i) {
            int j = nR.find(nL.q[i]);
            if (j < 0) continue;
            sq.push_back(nL.q[i]); sLi.push_back(int(i)); sRi.push_back(j); so.push_back(off);
            off += (long long)nL.dim[i] * nR.dim[j];
        }
        C.psi.ensure(size_t(std::max<long long>(off, 1)) * sizeof(double));
        GBD_CHECK_CUDA(cudaMemsetAsync(C.psi.p, 0, size_t(std::max<long long>(off, 1)) * sizeof(double), s));
        P.clear();
        for (size_t i = 0; i < nb.q.size(); ++i) {  // Q = new bond b+1 sector
            int si = H.sector_of(nb.q[i]);
            int eL = H.sL[si];
            for (const auto& sg1 : H.bL.segs[eL]) {   // s1, qp = Q - q_s1 at cut b
                Q qp = C.bonds[b].q[sg1.bq];
                auto it = std::lower_bound(sq.begin(), sq.end(), qp);
                if (it == sq.end() || *it != qp) continue;
                int ps = int(it - sq.begin());
                const Seg* sr = find_seg(nR, sRi[ps], sg1.s);
                int uo = Ap.out.find(qp);
                int ue = Ap.basis.find(qp);
                if (!sr || uo < 0 || ue < 0 || Ap.off[uo] < 0) continue;
                for (const auto& sg0 : Ap.basis.segs[ue]) {  // s0, cut-(b-1) sector
                    const Seg* sl = find_seg(nL, sLi[ps], sg0.s);
                    if (!sl) continue;
                    GemmTask t{};
                    int ldn = nR.dim[sRi[ps]];
                    t.C = C.psi.as<double>() + so[ps] + (long long)sl->off * ldn + sr->off;
                    t.ldc = ldn;
                    t.M = sg0.size;
                    t.N = nb.dim[i];
                    t.nbatch = 1;
                    t.beta = 0.0;
                    GemmSeg g{};
                    g.A = Ap.data.as<double>() + Ap.off[uo] + (long long)sg0.off * Ap.out.dim[uo];
                    g.lda = Ap.out.dim[uo];
                    g.B = Cbuf.as<double>() + coff[i] + (long long)sg1.off * nb.dim[i];
                    g.ldb = nb.dim[i];
                    g.K = sg1.size;
                    g.T = 1;
                    g.coef = 1.0;
                    P.add_task(t, {g});
                }
            }
        }
        P.check({{C.psi.p, C.psi.bytes}, {Cbuf.p, Cbuf.bytes}, {Ap.data.p, Ap.data.bytes}}, "truncate/next-");
        P.upload(s);
        P.launch(s);
        C.psi_b = b - 1;
        C.sites[b + 1] = std::move(I);
        C.site_kind[b + 1] = 1;
        C.envR[b + 1] = std::move(E);
    }
    GBD_CHECK_CUDA(cudaStreamSynchronize(s));
    (void)L;
    C.H = Heff();  // the enlarged operators belong to the old position
    return weight;
}

}  // namespace gbd
