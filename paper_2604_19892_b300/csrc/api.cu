// C ABI of the library (include/ipc.h): scene set-up, device memory, the
// Algorithm 1 driver that sequences the kernels, queries and the evaluation
// entry points.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "dev.cuh"
#include "host_mesh.h"
#include "ipc.h"
#include "kernels.h"

#include <atomic>

using namespace ipcb;

namespace {
std::atomic<long long> g_kernel_launches{0};
}

void ipcb::count_launch() { g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define CUDA_TRY(expr)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess) return fail(IPC_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int next_pow2(long long n) {
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}

struct Arena {
    ipc_alloc_fns fns{nullptr, nullptr, nullptr};
    std::vector<void*> ptrs;
    bool ok = true;
    size_t bytes = 0;
    void* get(size_t n) {
        if (!ok) return nullptr;  // no further requests once one has failed
        if (n == 0) n = 16;
        n = (n + 255) & ~(size_t)255;
        void* p = nullptr;
        if (fns.alloc) {
            p = fns.alloc(n, fns.ctx);
        } else if (cudaMalloc(&p, n) != cudaSuccess) {
            p = nullptr;
        }
        if (!p) {
            ok = false;
            return nullptr;
        }
        ptrs.push_back(p);
        bytes += n;
        return p;
    }
    template <class T>
    T* arr(size_t n) {
        return static_cast<T*>(get(n * sizeof(T)));
    }
    void put(void* p) {
        for (size_t i = 0; i < ptrs.size(); ++i)
            if (ptrs[i] == p) {
                if (fns.free)
                    fns.free(p, fns.ctx);
                else
                    cudaFree(p);
                ptrs[i] = ptrs.back();
                ptrs.pop_back();
                return;
            }
    }
    void release() {
        for (void* p : ptrs) {
            if (fns.free)
                fns.free(p, fns.ctx);
            else
                cudaFree(p);
        }
        ptrs.clear();
    }
};

// pinned host mirror of the device scalars plus contact counts
struct HostView {
    Scalars S;
    int nC, nCt;
    int cand_n[2];
    unsigned long long nonfinite;
};

}  // namespace

// CUDA-event stage timers: event pairs recorded on the step's stream and
// resolved after the next stream synchronisation.
struct StageProf {
    bool on = false;
    double ms[8] = {0};
    long long n[8] = {0};
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    struct Pending {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    cudaEvent_t get() {
        if (used == pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[used++];
    }
    void resolve() {
        for (auto& p : pending) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
                ms[p.stage] += t;
                n[p.stage] += 1;
            }
        }
        pending.clear();
        used = 0;
    }
    ~StageProf() {
        for (auto e : pool) cudaEventDestroy(e);
    }
};

struct ipc_scene {
    HostMesh hm;
    ipc_params prm;
    Arena arena;
    Dev<double> dd;
    Dev<float> df;
    int prec = IPC_PREC_FP64;
    HostView* hv = nullptr;  // pinned
    unsigned long long* nonfinite = nullptr;  // device counter of ipc_set_state's check
    std::vector<ipc_iter_record> trace;
    StageProf prof;
    // cached candidate pairs: built with margin cand_delta; cand_bound bounds
    // max_v |x_v - xref_v| of the current positions
    bool cand_ok = false;
    double cand_delta = 0.0;
    double cand_bound = 0.0;
    // CUDA graphs of the per-iteration launch sequences, keyed by the bytes of
    // the device-state struct (which changes with the buffer swaps) and the
    // sequence's host flags; a key is captured the second time it occurs
    std::unordered_map<unsigned long long, cudaGraphExec_t> graphs;
    std::unordered_set<unsigned long long> seen, uncapturable;
    // set once a RebuildMAS has been enqueued: the MAS blocks hold inverses
    bool mas_built = false;
    cudaStream_t own = nullptr;  // used when the caller passes the legacy default stream
    cudaEvent_t own_ev = nullptr;
    ~ipc_scene() {
        for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
        if (own_ev) cudaEventDestroy(own_ev);
        if (own) cudaStreamDestroy(own);
    }
};

namespace {

struct Stage {
    StageProf* p;
    int id;
    cudaStream_t st;
    cudaEvent_t b = nullptr;
    Stage(ipc_scene* s, int stage, cudaStream_t stream) : p(&s->prof), id(stage), st(stream) {
        if (!p->on) return;
        cudaEvent_t a = p->get();
        b = p->get();
        cudaEventRecord(a, st);
        p->pending.push_back({id, a, b});
    }
    ~Stage() {
        if (b) cudaEventRecord(b, st);
    }
};

template <class R>
Dev<R>& dev_of(ipc_scene* s);
template <>
Dev<double>& dev_of<double>(ipc_scene* s) {
    return s->dd;
}
template <>
Dev<float>& dev_of<float>(ipc_scene* s) {
    return s->df;
}

template <class T>
int upload(T* dst, const std::vector<T>& src, cudaStream_t st = 0) {
    if (src.empty()) return 0;
    CUDA_TRY(cudaMemcpyAsync(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, st));
    return 0;
}

ContactBuf alloc_contacts(Arena& A, int cap) {
    ContactBuf C;
    C.count = A.arr<int>(1);
    C.type = A.arr<int>(cap);
    C.v = A.arr<int4>(cap);
    C.key = A.arr<unsigned long long>(cap);
    C.d = A.arr<double>(cap);
    C.k = A.arr<double>(cap);
    C.bp = A.arr<double>(cap);
    C.r = A.arr<double>(3 * (size_t)cap);
    C.w = A.arr<double>(4 * (size_t)cap);
    return C;
}

template <class R>
int setup_dev(ipc_scene* s) {
    HostMesh& m = s->hm;
    Arena& A = s->arena;
    Dev<R>& D = dev_of<R>(s);
    memset(&D, 0, sizeof(D));
    const ipc_params& p = s->prm;
    D.nv = m.nv;
    D.nt = m.nt;
    D.nsv = (int)m.sv.size();
    D.nsf = (int)(m.sf.size() / 3);
    D.nse = (int)(m.se.size() / 2);
    D.nlev = m.nlev;
    D.ntp = (m.nt + kPack - 1) / kPack;
    int nb = 0;
    int coff = 0;
    for (int l = 0; l < m.nlev; ++l) {
        D.ngroups[l] = m.ngroups[l];
        D.nnodes[l] = m.nnodes[l];
        D.blk_off[l] = nb;
        nb += m.ngroups[l];
        D.coarse_off[l] = coff;
        if (l >= 1) coff += 3 * m.nnodes[l];
    }
    D.blk_off[m.nlev] = nb;
    D.coarse_off[m.nlev] = coff;
    D.cap = p.contact_capacity > 0 ? p.contact_capacity : std::max(4096, 16 * D.nsv + 16 * D.nse / 8);
    D.upd_cap = D.cap;
    D.straddle_cap = 32 * (D.nsf + D.nse) + 4096;  // 20 bytes per candidate
    D.h = p.h;
    D.piv32 = (float)(p.fp32_pivot_floor > 0.0 ? p.fp32_pivot_floor : 1e-6);
    D.dhat = p.dhat;
    D.kappa = p.kappa;
    D.eps_conv = p.tol * p.h * m.bbox_diag;
    D.delta = p.delta;
    D.cos_rot = std::cos(p.eps_rot_deg * M_PI / 180.0);
    D.ccd_shrink = p.ccd_shrink;
    D.eps_sing = p.eps_sing;
    D.eps_abs = p.eps_abs;
    D.K = p.K;
    D.ls_max = p.ls_max;
    D.wait_polls = p.wait_polls;
    {
        // rounding allowance of the energy check, tau = 64 u (|E_k| + 4 h^2
        // sum_t V_t mu_t): the second term is the size of the elastic terms
        // before they cancel near the rest state. u = 2^-52 for FP64
        // energies; with an FP32 bulk the elastic energy is double-float
        // from positions split to 2^-48 of their size, u = 2^-44 (a 16x
        // allowance for coordinates far from the origin relative to edges)
        double vmu = 0.0;
        for (int t = 0; t < m.nt; ++t) vmu += m.vol[t] * m.mu[t];
        const double u = sizeof(R) == 8 ? std::ldexp(1.0, -52) : std::ldexp(1.0, -44);
        D.tau_rel = 64.0 * u;
        D.tau_abs = 64.0 * u * 4.0 * p.h * p.h * vmu;
    }
    for (int r = 0; r < 3; ++r) {
        D.gravity[r] = m.gravity[r];
        D.gn[r] = m.gn[r];
    }
    D.has_ground = m.has_ground;
    D.goff = m.goff;
    // broad-phase cell: the mean surface edge, but no smaller than a third of
    // the longest one, so that on meshes mixing fine and coarse features
    // (thin spikes on a coarse ball) the coarse primitives still cover a few
    // cells each instead of falling into the list every query scans
    D.cell = std::max(std::max(m.mean_surface_edge, m.max_surface_edge / 3.0), 1e-12);

    const size_t n3 = 3 * (size_t)m.nv;
    // mesh
    std::vector<int4> tets(m.nt);
    for (int t = 0; t < m.nt; ++t) tets[t] = make_int4(m.tets[4 * t], m.tets[4 * t + 1], m.tets[4 * t + 2], m.tets[4 * t + 3]);
    int4* d_tets = A.arr<int4>(m.nt);
    std::vector<R> tb((size_t)D.ntp * 9 * kPack, (R)0);
    for (int t = 0; t < m.nt; ++t)
        for (int c = 0; c < 9; ++c) tb[(size_t)(t / kPack) * 9 * kPack + c * kPack + t % kPack] = (R)m.dminv[9 * (size_t)t + c];
    R* d_tb = A.arr<R>(tb.size());
    double* d_vol = A.arr<double>(m.nt);
    double* d_mu = A.arr<double>(m.nt);
    double* d_lam = A.arr<double>(m.nt);
    float2* d_ec = sizeof(R) == 4 ? A.arr<float2>(3 * (size_t)m.nt) : nullptr;
    std::vector<R> massr(m.mass.begin(), m.mass.end());
    R* d_mass = A.arr<R>(m.nv);
    double* d_massd = A.arr<double>(m.nv);
    int* d_sv = A.arr<int>(D.nsv);
    int* d_sf = A.arr<int>(m.sf.size());
    int* d_se = A.arr<int>(m.se.size());
    // hierarchy
    int* d_grp0 = A.arr<int>(m.nv);
    int* d_slot0 = A.arr<int>(m.nv);
    std::vector<int*> d_nov(m.nlev, nullptr), d_gon(m.nlev), d_son(m.nlev), d_mem(m.nlev);
    for (int l = 0; l < m.nlev; ++l) {
        if (l >= 1) d_nov[l] = A.arr<int>(m.nv);
        d_gon[l] = A.arr<int>(m.nnodes[l]);
        d_son[l] = A.arr<int>(m.nnodes[l]);
        d_mem[l] = A.arr<int>((size_t)m.ngroups[l] * kSub);
    }
    // state
    D.x = A.arr<double>(n3);
    D.xt = A.arr<double>(n3);
    D.xs = A.arr<double>(n3);
    D.xtry = A.arr<double>(n3);
    D.v = A.arr<double>(n3);
    D.g = A.arr<R>(n3);
    D.gtry = A.arr<R>(n3);
    D.z = A.arr<R>(n3);
    D.zprev = A.arr<R>(n3);
    D.p = A.arr<R>(n3);
    D.zp4 = A.arr<R>(8 * (size_t)m.nv);
    D.hess = A.arr<R>((size_t)D.ntp * kH * kPack);
    D.blocks = A.arr<R>((size_t)nb * kW);
    D.blocks16 = p.precision == IPC_PREC_BF16_MAS ? A.get((size_t)nb * kW16 * 2) : nullptr;
    D.jac = p.mas_mode == 3 ? A.arr<R>(9 * (size_t)m.nv) : nullptr;
    const int nb0 = m.nlev > 1 ? D.blk_off[1] : nb;
    D.asmb = A.arr<double>((size_t)nb0 * kBlk * kBlk);
    D.invflag = A.arr<int>(std::max(nb, 1));
    D.pivfix = A.arr<int>(1);
    D.asmbc = A.arr<double>((size_t)std::max(nb - nb0, 1) * kBlk * kBlk);
    D.pg_k = A.arr<double>((size_t)std::max(D.coarse_off[m.nlev] / 3, 1));
    // diagonal of each block's mass term: the lumped mass of the block's
    // nodes (sums of vertex masses at the coarse levels), fixed by the mesh
    std::vector<double> mdiag((size_t)nb * kBlk, 0.0);
    {
        std::vector<double> mnode;
        for (int l = 0; l < m.nlev; ++l) {
            mnode.assign(m.nnodes[l], 0.0);
            for (int v = 0; v < m.nv; ++v) mnode[l == 0 ? v : m.node_of_vert[l][v]] += (double)massr[v];
            for (int g = 0; g < m.ngroups[l]; ++g)
                for (int sl = 0; sl < kSub; ++sl) {
                    int n = m.members[l][(size_t)g * kSub + sl];
                    if (n < 0) continue;
                    for (int c = 0; c < 3; ++c) mdiag[((size_t)D.blk_off[l] + g) * kBlk + 3 * sl + c] = mnode[n];
                }
        }
    }
    double* d_mdiag = A.arr<double>(mdiag.size());
    D.mdiag = d_mdiag;
    // coarse elastic assembly contributions, fixed by the mesh: on every
    // coarse level, for every tet touching more than one node and every pair
    // of its node sets (P, Q) inside one group, the target (coarse block, node
    // slot i <= node slot j) and the tet's vertex masks of P (bits 0-3) and Q
    // (bits 4-7).
    // Sorted by target then tet; targets with many entries are cut into
    // chunks of at most kChunk summed separately (and added atomically).
    std::vector<int> tcon_off(m.nt + 1, 0);
    std::vector<int2> tcon;
    std::vector<int4> items;
    long long ncon = 0;
    {
        constexpr int kChunk = 64;
        struct Contrib {
            long long key;
            int t, masks;
        };
        std::vector<Contrib> cs;
        cs.reserve((size_t)m.nt * 14);
        for (int l = 1; l < m.nlev; ++l) {
            for (int t = 0; t < m.nt; ++t) {
                int nd[4], mk[4], nn = 0;
                for (int a = 0; a < 4; ++a) {
                    const int v = m.tets[4 * t + a];
                    const int n = m.node_of_vert[l][v];
                    int k = 0;
                    while (k < nn && nd[k] != n) ++k;
                    if (k == nn) {
                        nd[nn] = n;
                        mk[nn++] = 0;
                    }
                    mk[k] |= 1 << a;
                }
                if (nn < 2) continue;
                for (int i = 0; i < nn; ++i)
                    for (int j = i; j < nn; ++j) {
                        const int gi = m.group_of[l][nd[i]], gj = m.group_of[l][nd[j]];
                        if (gi != gj) continue;
                        int si = m.slot_of[l][nd[i]], sj = m.slot_of[l][nd[j]];
                        int mi = mk[i], mj = mk[j];
                        if (si > sj) {
                            std::swap(si, sj);
                            std::swap(mi, mj);
                        }
                        const long long key = ((long long)(D.blk_off[l] - D.blk_off[1] + gi) * kSub + si) * kSub + sj;
                        cs.push_back({key, t, mi | (mj << 4)});
                    }
            }
        }
        std::sort(cs.begin(), cs.end(), [](const Contrib& x, const Contrib& y) {
            return x.key != y.key ? x.key < y.key : x.t < y.t;
        });
        ncon = (long long)cs.size();
        for (const Contrib& c : cs) ++tcon_off[c.t + 1];
        for (int t = 0; t < m.nt; ++t) tcon_off[t + 1] += tcon_off[t];
        tcon.resize(cs.size());
        std::vector<int> cur(tcon_off.begin(), tcon_off.end() - 1);
        for (size_t e = 0; e < cs.size(); ++e) tcon[cur[cs[e].t]++] = make_int2((int)e, cs[e].masks);
        for (size_t e = 0; e < cs.size();) {
            size_t f = e;
            while (f < cs.size() && cs[f].key == cs[e].key) ++f;
            const long long k = cs[e].key;
            const int blk = (int)(k / (kSub * kSub)), si = (int)(k / kSub % kSub), sj = (int)(k % kSub);
            const int split = f - e > (size_t)kChunk ? 1 : 0;
            for (size_t c = e; c < f; c += kChunk) items.push_back(make_int4(blk, si, sj | (split << 8), (int)c));
            e = f;
        }
        items.push_back(make_int4(0, 0, 0, (int)cs.size()));
    }
    if (12 * ncon >= (1LL << 31)) return fail(IPC_ERR_CAPACITY, "scene: mesh too large for the assembly contribution list");
    int* d_tcon_off = A.arr<int>(tcon_off.size());
    int2* d_tcon = A.arr<int2>(std::max<size_t>(tcon.size(), 1));
    int4* d_items = A.arr<int4>(items.size());
    D.ncon = (int)ncon;
    D.nitem = (int)items.size() - 1;
    D.cval = A.arr<R>(std::max<size_t>(12 * (size_t)ncon, 1));
    D.tcon_off = d_tcon_off;
    D.tcon = d_tcon;
    D.item = d_items;
    D.coarse_r = A.arr<R>(std::max(coff, 1));
    D.coarse_y = A.arr<R>(std::max(coff, 1));
    D.C = alloc_contacts(A, D.cap);
    D.Ct = alloc_contacts(A, D.cap);
    D.Cb = alloc_contacts(A, D.cap);
    D.btab = next_pow2(2LL * D.cap);
    D.bkeys = A.arr<unsigned long long>(D.btab);
    D.bidx = A.arr<int>(D.btab);
    D.upd_c = A.arr<int>(D.upd_cap);
    D.upd_dS = A.arr<double>(D.upd_cap);
    D.upd_cnt = A.arr<int>(m.ngroups[0]);
    D.upd_off = A.arr<int>(m.ngroups[0] + 1);
    D.upd_cur = A.arr<int>(m.ngroups[0]);
    D.upd_list = A.arr<int>(4 * (size_t)D.upd_cap);
    D.topk = A.arr<int>((size_t)m.ngroups[0] * std::max(1, D.K));
    D.alpha = A.arr<double>(m.ngroups[0]);
    D.shrink = A.arr<double>(m.ngroups[0]);
    D.shrink3 = A.arr<double>(m.ngroups[0]);
    D.shrink4 = A.arr<double>(m.ngroups[0]);
    D.nbody = m.nbody;
    int* d_body = A.arr<int>(m.nv);
    D.body = d_body;
    D.alpha_b = A.arr<double>(m.nbody);
    D.shrink_b = A.arr<double>(m.nbody);
    D.shrink3_b = A.arr<double>(m.nbody);
    D.shrink4_b = A.arr<double>(m.nbody);
    D.vflags = A.arr<int>(32);
    D.str_v = A.arr<int4>(D.straddle_cap);
    D.str_t = A.arr<int>(D.straddle_cap);
    int nprim = std::max(std::max(D.nsf, D.nse), 1);
    D.nbuckets = next_pow2(std::max(4096, 2 * nprim));
    D.gcap = 32 * nprim + 4096;
    D.gcount = A.arr<int>(D.nbuckets + 1);
    D.gstart = A.arr<int>(D.nbuckets + 1);
    D.gfill = A.arr<int>(D.nbuckets);
    D.gbox = A.arr<float4>(2 * (size_t)D.gcap);
    D.gcell = A.arr<unsigned long long>(D.gcap);
    D.gtotal = A.arr<int>(1);
    D.glarge = A.arr<int>(nprim);
    D.gnlarge = A.arr<int>(1);
    D.gin = A.arr<int>(nprim);
    D.gtmp = A.arr<int>(std::max(D.nbuckets, m.ngroups[0]) / 1024 + 16);
    D.pbox = A.arr<float4>(2 * (size_t)nprim);
    D.xf = A.arr<float4>(m.nv);
    D.xsplit = sizeof(R) == 4 ? A.arr<float4>(2 * (size_t)m.nv) : nullptr;
    D.xpf = A.arr<float4>(m.nv);
    D.cellinv = A.arr<float>(1);
    D.cellsz = A.arr<double>(1);
    D.cand_cap = 48 * (D.nsv + D.nse) + 4096;
    D.xref = A.arr<double>(3 * (size_t)m.nv);
    D.cand_pt = A.arr<int2>(D.cand_cap);
    D.cand_ee = A.arr<int2>(D.cand_cap);
    D.cand_n = A.arr<int>(2);
    D.gpair_cap = p.grid_pair_capacity > 0 ? p.grid_pair_capacity : 16 * (D.nsv + D.nse) + 4096;
    D.gpair = A.arr<int2>(D.gpair_cap);
    D.gpair_n = A.arr<int>(2);
    D.S = A.arr<Scalars>(1);
    s->nonfinite = A.arr<unsigned long long>(1);
    if (!A.ok) return fail(IPC_ERR_OOM, "scene: device allocation failed");
    // level-0 assembly blocks are written at and below the diagonal only:
    // the entries above it are zeroed here, once
    CUDA_TRY(cudaMemset(D.asmb, 0, sizeof(double) * (size_t)nb0 * kBlk * kBlk));

    D.tets = d_tets;
    D.tetB = d_tb;
    D.tet_vol = d_vol;
    D.tet_mu = d_mu;
    D.tet_lam = d_lam;
    D.tet_ec = d_ec;
    D.mass = d_mass;
    D.massd = d_massd;
    D.sv = d_sv;
    D.sf = d_sf;
    D.se = d_se;
    D.grp0 = d_grp0;
    D.slot0 = d_slot0;
    for (int l = 0; l < m.nlev; ++l) {
        D.node_of_vert[l] = d_nov[l];
        D.grp_of_node[l] = d_gon[l];
        D.slot_of_node[l] = d_son[l];
        D.members[l] = d_mem[l];
    }
    CUDA_TRY(cudaMemcpy(d_tets, tets.data(), sizeof(int4) * m.nt, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_tb, tb.data(), sizeof(R) * tb.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_vol, m.vol.data(), sizeof(double) * m.nt, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_mu, m.mu.data(), sizeof(double) * m.nt, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_lam, m.lam.data(), sizeof(double) * m.nt, cudaMemcpyHostToDevice));
    if (d_ec) {
        // the elastic energy's coefficients as float pairs hi + lo (to ~2^-48)
        std::vector<float2> ec(3 * (size_t)m.nt);
        for (int t = 0; t < m.nt; ++t) {
            const double h2V = p.h * p.h * m.vol[t];
            const double c[3] = {0.5 * h2V * m.mu[t], h2V * m.mu[t], 0.5 * h2V * m.lam[t]};
            for (int k = 0; k < 3; ++k) {
                const float hi = (float)c[k];
                ec[3 * (size_t)t + k] = make_float2(hi, (float)(c[k] - (double)hi));
            }
        }
        CUDA_TRY(cudaMemcpy(d_ec, ec.data(), sizeof(float2) * ec.size(), cudaMemcpyHostToDevice));
    }
    CUDA_TRY(cudaMemcpy(d_mass, massr.data(), sizeof(R) * m.nv, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_massd, m.mass.data(), sizeof(double) * m.nv, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_mdiag, mdiag.data(), sizeof(double) * mdiag.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_tcon_off, tcon_off.data(), sizeof(int) * tcon_off.size(), cudaMemcpyHostToDevice));
    if (!tcon.empty()) CUDA_TRY(cudaMemcpy(d_tcon, tcon.data(), sizeof(int2) * tcon.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
    if (D.nsv) CUDA_TRY(cudaMemcpy(d_sv, m.sv.data(), sizeof(int) * D.nsv, cudaMemcpyHostToDevice));
    if (D.nsf) CUDA_TRY(cudaMemcpy(d_sf, m.sf.data(), sizeof(int) * m.sf.size(), cudaMemcpyHostToDevice));
    if (D.nse) CUDA_TRY(cudaMemcpy(d_se, m.se.data(), sizeof(int) * m.se.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_grp0, m.group_of[0].data(), sizeof(int) * m.nv, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_slot0, m.slot_of[0].data(), sizeof(int) * m.nv, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_body, m.body.data(), sizeof(int) * m.nv, cudaMemcpyHostToDevice));
    for (int l = 0; l < m.nlev; ++l) {
        if (l >= 1) CUDA_TRY(cudaMemcpy(d_nov[l], m.node_of_vert[l].data(), sizeof(int) * m.nv, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(d_gon[l], m.group_of[l].data(), sizeof(int) * m.nnodes[l], cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(d_son[l], m.slot_of[l].data(), sizeof(int) * m.nnodes[l], cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(d_mem[l], m.members[l].data(), sizeof(int) * m.members[l].size(), cudaMemcpyHostToDevice));
    }
    CUDA_TRY(cudaMemcpy(D.x, m.x0.data(), sizeof(double) * n3, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(D.v, m.v0.data(), sizeof(double) * n3, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemset(D.S, 0, sizeof(Scalars)));
    CUDA_TRY(cudaMemset(D.invflag, 0, sizeof(int) * std::max(D.blk_off[D.nlev], 1)));
    CUDA_TRY(cudaMemset(D.pivfix, 0, sizeof(int)));
    CUDA_TRY(cudaMemset(D.hess, 0, sizeof(R) * (size_t)D.ntp * kH * kPack));
    CUDA_TRY(cudaMemset(D.Cb.count, 0, sizeof(int)));
    CUDA_TRY(cudaMemset(D.C.count, 0, sizeof(int)));
    CUDA_TRY(cudaMemset(D.Ct.count, 0, sizeof(int)));
    // set-up work runs on the legacy stream and is waited for there, not by
    // a device-wide synchronisation: other scenes may be stepping, and
    // capturing CUDA graphs, on non-blocking streams of other threads
    CUDA_TRY(cudaStreamSynchronize(cudaStreamLegacy));
    // launch configuration of the per-iteration block apply, timed on this
    // scene's block count (the autotuner; its values are overwritten by the
    // first RebuildMAS)
    if (p.apply_ctas > 0)
        D.apply_ctas = p.apply_ctas;
    else
        autotune_apply(D, (cudaStream_t)0);
    CUDA_TRY(cudaStreamSynchronize(cudaStreamLegacy));
    CUDA_TRY(cudaMemset(D.S, 0, sizeof(Scalars)));
    return 0;
}

// Launches seq() on st as a CUDA graph when the scene allows it: replayed
// when this key (device-state bytes, variant) has a graph, captured when the
// key is seen for the second time (the first run warms one-time setup and
// allocations), launched directly otherwise. A sequence that cannot be
// captured is launched directly from then on.
template <class R, class F>
int run_seq(ipc_scene* s, const Dev<R>& D, cudaStream_t st, unsigned long long variant, F&& seq) {
    if (!s->prm.graphs || s->prof.on) {
        seq();
        return 0;
    }
    unsigned long long key = 1469598103934665603ULL ^ (variant * 0x9E3779B97F4A7C15ULL);
    const unsigned char* b = reinterpret_cast<const unsigned char*>(&D);
    for (size_t i = 0; i < sizeof(Dev<R>); ++i) key = (key ^ b[i]) * 1099511628211ULL;
    auto it = s->graphs.find(key);
    if (it != s->graphs.end()) {
        CUDA_TRY(cudaGraphLaunch(it->second, st));
        return 0;
    }
    if (s->uncapturable.count(key) || s->seen.insert(key).second) {
        seq();
        return 0;
    }
    if (s->graphs.size() >= 64) {  // bound the cache (buffers regrown many times)
        for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
        s->graphs.clear();
    }
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        seq();
        if (cudaStreamEndCapture(st, &g) == cudaSuccess && g &&
            cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
            cudaGraphDestroy(g);
            s->graphs[key] = ex;
            CUDA_TRY(cudaGraphLaunch(ex, st));
            return 0;
        }
        if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();  // clear the capture failure
    s->uncapturable.insert(key);
    seq();  // nothing of the failed capture ran
    return 0;
}

template <class R>
int read_view(ipc_scene* s, const Dev<R>& D, cudaStream_t st) {
    CUDA_TRY(cudaMemcpyAsync(&s->hv->S, D.S, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&s->hv->nC, D.C.count, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&s->hv->nCt, D.Ct.count, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (s->prof.on) s->prof.resolve();
    return 0;
}

template <class T>
__global__ void k_count_nonfinite(const T* a, size_t n, unsigned long long* out) {
    unsigned long long c = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double v = (double)a[i];
        if (!(v == v) || v - v != 0.0) ++c;
    }
    if (c) atomicAdd(out, c);
}

// Describe where non-finite values sit (for the error message of a NaN stop).
template <class R>
std::string nonfinite_report(const Dev<R>& D, const Scalars& S, cudaStream_t st) {
    unsigned long long* cnt = nullptr;
    if (cudaMalloc(&cnt, 8 * sizeof(unsigned long long)) != cudaSuccess) return "";
    cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), st);
    size_t n3 = 3 * (size_t)D.nv;
    size_t nb = (size_t)D.blk_off[D.nlev] * kW;
    const size_t nbsq = (size_t)D.blk_off[D.nlev] * kBlk * kBlk;
    KL(k_count_nonfinite<R><<<256, 256, 0, st>>>(D.g, n3, cnt + 0));
    KL(k_count_nonfinite<R><<<256, 256, 0, st>>>(D.z, n3, cnt + 1));
    KL(k_count_nonfinite<R><<<256, 256, 0, st>>>(D.p, n3, cnt + 2));
    KL(k_count_nonfinite<R><<<256, 256, 0, st>>>(D.blocks, nb, cnt + 3));
    KL(k_count_nonfinite<R><<<256, 256, 0, st>>>(D.hess, (size_t)D.ntp * kH * kPack, cnt + 4));
    KL(k_count_nonfinite<double><<<256, 256, 0, st>>>(D.x, n3, cnt + 5));
    const size_t nb0 = (size_t)(D.nlev > 1 ? D.blk_off[1] : D.blk_off[D.nlev]) * kBlk * kBlk;
    KL(k_count_nonfinite<double><<<256, 256, 0, st>>>(D.asmb, nb0, cnt + 6));
    if (nbsq > nb0) KL(k_count_nonfinite<double><<<256, 256, 0, st>>>(D.asmbc, nbsq - nb0, cnt + 7));
    unsigned long long h[8] = {0};
    cudaMemcpyAsync(h, cnt, sizeof h, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    cudaFree(cnt);
    char buf[512];
    snprintf(buf, sizeof buf,
             " (non-finite: g %llu, z %llu, p %llu, blocks %llu, tet Hessians %llu, x %llu, assembled %llu; "
             "gz %g zHz %g zHp %g pHp %g gp %g mu %g nu %g; first non-finite block %d with %d updates: "
             "max|rhs| %g max|Y| %g max|lambda| %g max dS %g)",
             h[0], h[1], h[2], h[3], h[4], h[5], h[6], S.gz, S.zHz, S.zHp, S.pHp, S.gp, S.mu, S.nu, S.dbg_block,
             S.dbg_ns, S.dbg_rhs, S.dbg_y, S.dbg_lam, S.dbg_ds);
    return buf;
}

template <class R>
__global__ void k_velocity(Dev<R> D) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * D.nv) return;
    D.v[i] = (D.x[i] - D.xs[i]) / D.h;
}

template <class R>
__global__ void k_set_scalar_double(double* dst, double v) {
    *dst = v;
}

template <class R>
__global__ void k_reset_flags(Dev<R> D) {
    D.S->overflow = 0;
    D.S->nan_flag = 0;
    D.S->async_timeout = 0;
    D.S->dbg_block = -1;
}

// contacts, energy and gradient at D.x into C / g / E_k
template <class R>
void eval_current(const Dev<R>& D, cudaStream_t st, bool list = false) {
    if (list)
        launch_detect_list(D, D.x, D.C, st);
    else
        launch_detect(D, D.x, D.C, st);
    launch_energy_grad(D, D.x, D.C, D.g, &D.S->E_k, st);
}

template <class R>
void eval_trial(const Dev<R>& D, int mode, double c, cudaStream_t st, bool list = false) {
    launch_trial_positions(D, mode, c, st);
    if (list)
        launch_detect_list(D, D.xtry, D.Ct, st);
    else
        launch_detect(D, D.xtry, D.Ct, st);
    launch_energy_grad(D, D.xtry, D.Ct, D.gtry, &D.S->E_try, st);
    launch_accept(D, st);
}

// Builds the candidate lists at x with margin delta; grows them (up to
// max_pairs entries each) when they fill up. Returns 1 when the lists hold
// every candidate, 0 when they would need more than max_pairs, < 0 on error.
template <class R>
int build_lists(ipc_scene* s, Dev<R>& D, const double* x, double delta, long long max_pairs, cudaStream_t st) {
    for (int attempt = 0; attempt < 4; ++attempt) {
        launch_cand_build(D, x, delta, st);
        CUDA_TRY(cudaMemcpyAsync(s->hv->cand_n, D.cand_n, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        // the append counters stop at the capacity, so a full list may have
        // dropped pairs: grow 4x and rebuild
        if (std::max(s->hv->cand_n[0], s->hv->cand_n[1]) < D.cand_cap) return 1;
        if (D.cand_cap >= max_pairs) return 0;
        long long cap = std::min(max_pairs, 4LL * D.cand_cap);
        int2* a = s->arena.arr<int2>(cap);
        int2* b = s->arena.arr<int2>(cap);
        if (!a || !b) {
            if (a) s->arena.put(a);
            if (b) s->arena.put(b);
            s->arena.ok = true;
            return 0;
        }
        s->arena.put(D.cand_pt);
        s->arena.put(D.cand_ee);
        D.cand_pt = a;
        D.cand_ee = b;
        D.cand_cap = (int)cap;
    }
    return 0;
}

// Broad phase of this iteration. The cached candidate lists serve while
// every position of the CCD segment stays within cand_delta of the build
// positions: max_v |x_v - xref_v| + max_v |p_v| <= delta. Otherwise they
// are rebuilt here at x_k with delta = max(2 dhat, 2 max|p|) when the
// direction is short (max|p| <= 2 dhat); long directions (the first
// iterations of a timestep) use the per-call hashed grid.
template <class R>
int choose_broad_phase(ipc_scene* s, Dev<R>& D, cudaStream_t st, bool* use_list, double* bound_after) {
    const double pm = s->hv->S.pmax, md = s->hv->S.maxdisp;
    const int mode = s->prm.broad_phase;
    *use_list = false;
    *bound_after = INFINITY;
    if (mode == 1) return IPC_OK;
    if (s->cand_ok && md + pm <= s->cand_delta) {
        *use_list = true;
        *bound_after = md + pm;
        return IPC_OK;
    }
    if (pm <= 2.0 * D.dhat || mode == 2) {
        const double delta = std::max(2.0 * D.dhat, 2.0 * pm);
        const long long lim = mode == 2 ? (1LL << 30) : 256LL * (D.nsv + D.nse) + 4096;
        int r = build_lists(s, D, D.x, delta, lim, st);
        if (r < 0) return r;
        s->cand_ok = r == 1;
        if (s->cand_ok) {
            s->cand_delta = delta;
            *use_list = true;
            *bound_after = pm;
        }
    }
    return IPC_OK;
}

// Algorithm 1 for one timestep.
template <class R>
int run_timestep(ipc_scene* s, cudaStream_t st, ipc_step_stats* acc) {
    Dev<R>& D = dev_of<R>(s);
    const ipc_params& P = s->prm;
    const size_t n3 = 3 * (size_t)D.nv;
    {
        Stage t(s, 7, st);
        KL(k_reset_flags<R><<<1, 1, 0, st>>>(D));
        launch_predict(D, st);
        CUDA_TRY(cudaMemsetAsync(D.zprev, 0, sizeof(R) * n3, st));
        CUDA_TRY(cudaMemsetAsync(D.p, 0, sizeof(R) * n3, st));
        eval_current(D, st, s->prm.broad_phase != 1 && s->cand_ok && s->cand_bound <= s->cand_delta);
    }
    if (int e = read_view(s, D, st)) return e;
    if (s->hv->S.overflow & 1) return fail(IPC_ERR_CAPACITY, "contact buffer overflow");
    if (s->hv->S.nonpos)
        return fail(IPC_ERR_INTERSECTING, "a contact has non-positive distance");
    // an energy that overflowed (e.g. velocities so large that |x - x~|^2
    // exceeds the FP64 range) stops the timestep before any kernel uses it;
    // x is left as it was
    if (!std::isfinite(s->hv->S.E_k))
        return fail(IPC_ERR_NUMERIC, "non-finite energy at the start of the timestep");
    s->trace.clear();
    double Ek = s->hv->S.E_k;
    double min_dist = s->hv->S.min_dist;
    bool restart = true;
    int k = 0, converged = 0, restarts = 0, halvings = 0, failures = 0, fallbacks = 0;
    double znorm = 0.0;
    for (k = 0; k < P.iter_max; ++k) {
        ipc_iter_record rec;
        memset(&rec, 0, sizeof rec);
        rec.restart = restart ? 1 : 0;
        rec.n_contacts = s->hv->nC;
        // MAS maintenance between restarts: Woodbury updates, a full rebuild
        // (the blocks and H_base at the current state; not a PNCG restart) or
        // nothing (frozen)
        // (mas_mode 3, block-Jacobi, is rebuilt at restarts like MAS and frozen
        // between them)
        const bool rebuild = restart || P.mas_mode == 1;
        const bool woodbury = !restart && P.mas_mode == 0;
        if (rebuild) {
            ++restarts;
            s->mas_built = true;
        }
        run_seq(s, D, st, restart ? 1 : (P.mas_mode == 1 ? 5 : P.mas_mode == 2 ? 6 : 2), [&] {
            if (rebuild) {
                Stage t(s, 0, st);
                launch_restart(D, D.x, D.C, st);
            } else if (woodbury) {
                Stage t(s, 1, st);
                launch_classify(D, D.C, st);
            }
            {
                Stage t(s, 7, st);
                launch_restrict(D, D.g, st);
            }
            {
                Stage t(s, 2, st);
                launch_blocks(D, D.g, D.z, D.C, woodbury, st);
            }
            {
                Stage t(s, 7, st);
                launch_prolong(D, D.z, st);
            }
            {
                Stage t(s, 3, st);
                launch_forms(D, D.C, restart, st);
            }
            {
                Stage t(s, 4, st);
                launch_direction(D, restart, st);
            }
            // g.z, max|p|, the list drift and the bulk-copy status of this
            // iteration
            cudaMemcpyAsync(&s->hv->S.gz, &D.S->gz, sizeof(double), cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(&s->hv->S.pmax, &D.S->pmax, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(&s->hv->S.async_timeout, &D.S->async_timeout, sizeof(int), cudaMemcpyDeviceToHost, st);
        });
        bool use_list = false;
        double bound_after = INFINITY;
        CUDA_TRY(cudaStreamSynchronize(st));
        // z is not defined after a timed-out block copy: stop before it is used
        if (s->hv->S.async_timeout) return fail(IPC_ERR_TIMEOUT, "a bulk copy into shared memory did not complete");
        if (!restart && !(s->hv->S.gz > 0.0)) {
            // the Woodbury-patched preconditioner is not positive at g (FP32
            // inverses of very stiff blocks): no step; the iteration is
            // redone as a restart with freshly inverted blocks
            rec.gz = s->hv->S.gz;
            rec.energy_before = rec.energy_after = Ek;
            rec.r = INFINITY;
            s->trace.push_back(rec);
            restart = true;
            continue;
        }
        {
            Stage t(s, 5, st);
            if (int e = choose_broad_phase(s, D, st, &use_list, &bound_after)) return e;
            if (use_list) {
                run_seq(s, D, st, 3, [&] { launch_ccd_list(D, st, 1); });
                launch_ccd_list(D, st, 2);
            } else {
                launch_ccd(D, st);
            }
            if (P.ccd_mode == 1) launch_global_alpha(D, st);  // one step for every subdomain
        }
        if (use_list) {
            run_seq(s, D, st, 4, [&] {
                {
                    Stage t(s, 6, st);
                    eval_trial(D, 0, 0.0, st, true);
                }
                cudaMemcpyAsync(&s->hv->S, D.S, sizeof(Scalars), cudaMemcpyDeviceToHost, st);
                cudaMemcpyAsync(&s->hv->nC, D.C.count, sizeof(int), cudaMemcpyDeviceToHost, st);
                cudaMemcpyAsync(&s->hv->nCt, D.Ct.count, sizeof(int), cudaMemcpyDeviceToHost, st);
            });
            CUDA_TRY(cudaStreamSynchronize(st));
            if (s->prof.on) s->prof.resolve();
        } else {
            {
                Stage t(s, 6, st);
                eval_trial(D, 0, 0.0, st, false);
            }
            if (int e = read_view(s, D, st)) return e;
        }
        Scalars S = s->hv->S;
        if (S.async_timeout) return fail(IPC_ERR_TIMEOUT, "a bulk copy into shared memory did not complete");
        if (S.nan_flag || !(S.gz == S.gz))
            return fail(IPC_ERR_NUMERIC, "NaN in the PNCG iteration at iteration " + std::to_string(k) +
                                             (restart ? " (restart)" : "") + nonfinite_report(D, S, st));
        if (S.overflow & 1) return fail(IPC_ERR_CAPACITY, "contact buffer overflow");
        if (S.ccd_passes < 0) ++fallbacks;
        rec.n_update = S.n_upd;
        rec.mu = S.mu;
        rec.nu = S.nu;
        rec.gz = S.gz;
        rec.znorm = S.znorm;
        rec.alpha_min = S.alpha_min;
        rec.alpha_max = S.alpha_max;
        rec.pmax = S.pmax;
        rec.ccd_passes = S.ccd_passes;
        rec.ccd_passes_body = S.ccd_passes_b;
        rec.cached_pairs = use_list ? 1 : 0;
        rec.energy_before = Ek;
        int accepted = S.accepted;
        int halv = 0;
        if (!accepted) {
            // trial list after the per-subdomain step: per-body steps scaled
            // by 1, 1/2, 1/4, 1/8 (when some body exceeds the uniform step),
            // then the uniform step alpha_min / 2^j. When the first trial
            // already was the per-body step (the per-subdomain verification
            // fell back, the per-body one did not: k_trial), the per-body
            // tier goes on at 1/2
            halv = 1;
            const bool body_tier = S.alpha_bmax > S.alpha_min;
            const bool body_first = body_tier && S.ccd_passes < 0 && S.ccd_passes_b >= 0;
            const int nbt = body_tier ? (body_first ? 3 : 4) : 0;
            const int j0 = (S.alpha_max > S.alpha_min || body_tier) ? 0 : 1;
            for (int ls = 1; ls <= P.ls_max; ++ls) {
                {
                    Stage t(s, 6, st);
                    if (ls <= nbt)
                        eval_trial(D, 1, std::ldexp(1.0, -(ls - (body_first ? 0 : 1))), st, use_list);
                    else
                        eval_trial(D, 2, std::ldexp(S.alpha_min, -(j0 + ls - 1 - nbt)), st, use_list);
                }
                if (int e = read_view(s, D, st)) return e;
                if (s->hv->S.overflow & 1) return fail(IPC_ERR_CAPACITY, "contact buffer overflow");
                if (s->hv->S.accepted) {
                    accepted = 1;
                    break;
                }
                ++halv;
            }
        }
        rec.ls_halvings = halv;
        halvings += halv;
        // bound on max_v |x_v - xref_v| for the next iteration or timestep
        if (use_list)
            s->cand_bound = accepted ? bound_after : bound_after - s->hv->S.pmax;
        else
            s->cand_bound = INFINITY;
        if (accepted) {
            std::swap(D.x, D.xtry);
            std::swap(D.C, D.Ct);
            std::swap(D.g, D.gtry);
            Ek = s->hv->S.E_k;
            s->hv->nC = s->hv->nCt;
            min_dist = s->hv->S.min_dist;
        }
        rec.energy_after = Ek;
        znorm = S.znorm;
        rec.r = S.gz > 0.0 ? std::fabs(S.gzprev) / S.gz : INFINITY;
        bool forced = !accepted;
        if (forced) ++failures;
        s->trace.push_back(rec);
        // Algorithm 1 tests convergence after the update whatever it was: a
        // restart iteration with |z| <= eps ends the timestep converged even
        // when no trial was accepted (what is left is below the tolerance)
        if (restart && S.znorm <= D.eps_conv) {
            converged = 1;
            ++k;
            break;
        }
        if (forced && restart) {
            ++k;
            break;
        }
        restart = forced || !(rec.r <= D.delta) || S.znorm <= D.eps_conv;
        std::swap(D.z, D.zprev);
    }
    KL(k_velocity<R><<<(int)((n3 + 255) / 256), 256, 0, st>>>(D));
    CUDA_TRY(cudaGetLastError());
    acc->steps += 1;
    acc->iters += k;
    acc->restarts += restarts;
    acc->ls_halvings += halvings;
    acc->ls_failures += failures;
    acc->converged = converged;
    acc->ccd_fallbacks += fallbacks;
    acc->n_contacts = s->hv->nC;
    acc->energy = Ek;
    acc->min_dist = min_dist;
    acc->znorm = znorm;
    return converged ? IPC_OK : IPC_NOT_CONVERGED;
}

template <class R>
int step_impl(ipc_scene* s, int n, cudaStream_t caller, ipc_step_stats* out) {
    // CUDA graphs cannot be captured on the legacy default stream: the work
    // then runs on a stream of the scene's own, after everything queued on
    // the caller's stream and before anything queued there later
    cudaStream_t st = caller;
    if (caller == nullptr || caller == cudaStreamLegacy) {
        if (!s->own) {
            CUDA_TRY(cudaStreamCreateWithFlags(&s->own, cudaStreamNonBlocking));
            CUDA_TRY(cudaEventCreateWithFlags(&s->own_ev, cudaEventDisableTiming));
        }
        CUDA_TRY(cudaEventRecord(s->own_ev, caller));
        CUDA_TRY(cudaStreamWaitEvent(s->own, s->own_ev, 0));
        st = s->own;
    }
    ipc_step_stats acc;
    memset(&acc, 0, sizeof acc);
    int worst = IPC_OK;
    int rc = IPC_OK;
    for (int i = 0; i < n; ++i) {
        int r = run_timestep<R>(s, st, &acc);
        if (r < 0) {
            rc = r;
            break;
        }
        if (r > worst) worst = r;
    }
    if (st != caller) {
        cudaEventRecord(s->own_ev, st);
        cudaStreamWaitEvent(caller, s->own_ev, 0);
    }
    if (out) *out = acc;
    if (rc < 0) return rc;
    CUDA_TRY(cudaStreamSynchronize(st));
    CUDA_TRY(cudaGetLastError());
    return worst;
}

template <class R>
std::vector<R> to_r(const double* a, size_t n) {
    std::vector<R> v(n);
    for (size_t i = 0; i < n; ++i) v[i] = (R)a[i];
    return v;
}

template <class R>
int eval_energy_impl(ipc_scene* s, const double* x, const double* xt, double* E, double* g, cudaStream_t st) {
    Dev<R>& D = dev_of<R>(s);
    size_t n3 = 3 * (size_t)D.nv;
    CUDA_TRY(cudaMemcpyAsync(D.xtry, x, sizeof(double) * n3, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(D.xt, xt, sizeof(double) * n3, cudaMemcpyHostToDevice, st));
    KL(k_reset_flags<R><<<1, 1, 0, st>>>(D));
    launch_detect(D, D.xtry, D.Ct, st);
    launch_energy_grad(D, D.xtry, D.Ct, g ? D.gtry : (R*)nullptr, &D.S->E_try, st);
    if (int e = read_view(s, D, st)) return e;
    if (s->hv->S.overflow & 1) return fail(IPC_ERR_CAPACITY, "contact buffer overflow");
    if (E) *E = s->hv->S.E_try;
    if (g) {
        std::vector<R> gr(n3);
        CUDA_TRY(cudaMemcpy(gr.data(), D.gtry, sizeof(R) * n3, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n3; ++i) g[i] = (double)gr[i];
    }
    return IPC_OK;
}

template <class R>
int eval_contacts_impl(ipc_scene* s, const double* x, int cap, int* n, int* type, int* ids, int* verts, double* dist,
                       double* kk, double* grad12, cudaStream_t st) {
    Dev<R>& D = dev_of<R>(s);
    size_t n3 = 3 * (size_t)D.nv;
    CUDA_TRY(cudaMemcpyAsync(D.xtry, x, sizeof(double) * n3, cudaMemcpyHostToDevice, st));
    KL(k_reset_flags<R><<<1, 1, 0, st>>>(D));
    if (s->prm.broad_phase == 2) {
        // candidate lists built at x itself (margin 2 dhat)
        s->cand_ok = false;
        int r = build_lists(s, D, D.xtry, 2.0 * D.dhat, 1LL << 30, st);
        if (r < 0) return r;
        if (r == 0) return fail(IPC_ERR_CAPACITY, "candidate list overflow");
        launch_detect_list(D, D.xtry, D.Ct, st);
    } else {
        launch_detect(D, D.xtry, D.Ct, st);
    }
    if (int e = read_view(s, D, st)) return e;
    if (s->hv->S.overflow & 1) return fail(IPC_ERR_CAPACITY, "contact buffer overflow");
    int nc = std::min(s->hv->nCt, D.cap);
    if (n) *n = nc;
    int m = std::min(nc, cap);
    if (m <= 0) return IPC_OK;
    std::vector<int> ty(m);
    std::vector<int4> vv(m);
    std::vector<unsigned long long> key(m);
    std::vector<double> d(m), k(m), r(3 * (size_t)m), w(4 * (size_t)m);
    CUDA_TRY(cudaMemcpy(ty.data(), D.Ct.type, sizeof(int) * m, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(vv.data(), D.Ct.v, sizeof(int4) * m, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(key.data(), D.Ct.key, sizeof(unsigned long long) * m, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(d.data(), D.Ct.d, sizeof(double) * m, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(k.data(), D.Ct.k, sizeof(double) * m, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(r.data(), D.Ct.r, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(w.data(), D.Ct.w, sizeof(double) * 4 * m, cudaMemcpyDeviceToHost));
    for (int i = 0; i < m; ++i) {
        if (type) type[i] = ty[i];
        if (ids) {
            ids[2 * i] = (int)((key[i] >> 31) & 0x7FFFFFFFULL);
            ids[2 * i + 1] = (int)(key[i] & 0x7FFFFFFFULL);
        }
        if (verts) {
            verts[4 * i] = vv[i].x;
            verts[4 * i + 1] = vv[i].y;
            verts[4 * i + 2] = vv[i].z;
            verts[4 * i + 3] = vv[i].w;
        }
        if (dist) dist[i] = d[i];
        if (kk) kk[i] = k[i];
        if (grad12)
            for (int j = 0; j < 4; ++j)
                for (int c = 0; c < 3; ++c) grad12[12 * i + 3 * j + c] = (ty[i] == 2 && j > 0) ? 0.0 : w[4 * i + j] * r[3 * i + c];
    }
    return IPC_OK;
}

// restart at x_base into C, optional classification of the contacts at
// x_curr (into Ct); returns the buffer holding the classified contacts
template <class R>
int prepare_precond(ipc_scene* s, const double* x_base, const double* x_curr, cudaStream_t st, bool* wood) {
    Dev<R>& D = dev_of<R>(s);
    size_t n3 = 3 * (size_t)D.nv;
    Dev<R> E = D;  // evaluation view: positions in scratch buffers
    E.x = D.xtry;
    CUDA_TRY(cudaMemcpyAsync(D.xtry, x_base, sizeof(double) * n3, cudaMemcpyHostToDevice, st));
    KL(k_reset_flags<R><<<1, 1, 0, st>>>(D));
    launch_detect(E, E.x, E.C, st);
    launch_restart(E, E.x, E.C, st);
    s->mas_built = true;
    *wood = false;
    if (x_curr) {
        CUDA_TRY(cudaMemcpyAsync(D.xs, x_curr, sizeof(double) * n3, cudaMemcpyHostToDevice, st));
        launch_detect(E, D.xs, E.Ct, st);
        launch_classify(E, E.Ct, st);
        *wood = true;
    }
    if (int e = read_view(s, D, st)) return e;
    if (s->hv->S.overflow) return fail(IPC_ERR_CAPACITY, "buffer overflow in evaluation");
    return IPC_OK;
}

template <class R>
int eval_precond_impl(ipc_scene* s, const double* xb, const double* xc, const double* g, double* z, cudaStream_t st) {
    Dev<R>& D = dev_of<R>(s);
    size_t n3 = 3 * (size_t)D.nv;
    bool wood;
    if (int e = prepare_precond<R>(s, xb, xc, st, &wood)) return e;
    std::vector<R> gr = to_r<R>(g, n3);
    CUDA_TRY(cudaMemcpyAsync(D.g, gr.data(), sizeof(R) * n3, cudaMemcpyHostToDevice, st));
    launch_precond(D, D.g, D.z, wood ? D.Ct : D.C, wood, st);
    std::vector<R> zr(n3);
    CUDA_TRY(cudaMemcpyAsync(zr.data(), D.z, sizeof(R) * n3, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&s->hv->S.async_timeout, &D.S->async_timeout, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (s->hv->S.async_timeout) return fail(IPC_ERR_TIMEOUT, "a bulk copy into shared memory did not complete");
    for (size_t i = 0; i < n3; ++i) z[i] = (double)zr[i];
    return IPC_OK;
}

template <class R>
int eval_forms_impl(ipc_scene* s, const double* xb, const double* xc, const double* z, const double* p, double out[3],
                    cudaStream_t st) {
    Dev<R>& D = dev_of<R>(s);
    size_t n3 = 3 * (size_t)D.nv;
    bool wood;
    if (int e = prepare_precond<R>(s, xb, xc, st, &wood)) return e;
    std::vector<R> zr = to_r<R>(z, n3), pr = to_r<R>(p, n3);
    CUDA_TRY(cudaMemcpyAsync(D.z, zr.data(), sizeof(R) * n3, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(D.p, pr.data(), sizeof(R) * n3, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemsetAsync(D.g, 0, sizeof(R) * n3, st));
    CUDA_TRY(cudaMemsetAsync(D.zprev, 0, sizeof(R) * n3, st));
    launch_forms(D, wood ? D.Ct : D.C, false, st);
    if (int e = read_view(s, D, st)) return e;
    out[0] = s->hv->S.zHz;
    out[1] = s->hv->S.zHp;
    out[2] = s->hv->S.pHp;
    return IPC_OK;
}

template <class R>
int eval_ccd_impl(ipc_scene* s, const double* x, const double* p, double* alpha, int* passes, double* alpha_body,
                  int* passes_body, cudaStream_t st) {
    Dev<R>& D = dev_of<R>(s);
    size_t n3 = 3 * (size_t)D.nv;
    Dev<R> E = D;
    E.x = D.xtry;
    CUDA_TRY(cudaMemcpyAsync(D.xtry, x, sizeof(double) * n3, cudaMemcpyHostToDevice, st));
    std::vector<R> pr = to_r<R>(p, n3);
    CUDA_TRY(cudaMemcpyAsync(D.p, pr.data(), sizeof(R) * n3, cudaMemcpyHostToDevice, st));
    double pm = 0.0;
    for (int v = 0; v < D.nv; ++v) {
        double a = (double)pr[3 * v], b = (double)pr[3 * v + 1], c = (double)pr[3 * v + 2];
        pm = std::max(pm, std::sqrt(a * a + b * b + c * c));
    }
    KL(k_set_scalar_double<R><<<1, 1, 0, st>>>(&D.S->pmax, pm));
    KL(k_reset_flags<R><<<1, 1, 0, st>>>(D));
    if (s->prm.broad_phase == 2) {
        // candidate lists built at x with a margin covering the segment
        s->cand_ok = false;
        int r = build_lists(s, D, D.xtry, std::max(2.0 * D.dhat, 2.0 * pm), 1LL << 30, st);
        if (r < 0) return r;
        if (r == 0) return fail(IPC_ERR_CAPACITY, "candidate list overflow");
        E.cand_pt = D.cand_pt;
        E.cand_ee = D.cand_ee;
        E.cand_cap = D.cand_cap;
        launch_ccd_list(E, st);
    } else {
        launch_ccd(E, st);
    }
    if (int e = read_view(s, D, st)) return e;
    int ng = D.ngroups[0];
    CUDA_TRY(cudaMemcpy(alpha, D.alpha, sizeof(double) * ng, cudaMemcpyDeviceToHost));
    if (passes) *passes = s->hv->S.ccd_passes;
    if (alpha_body) CUDA_TRY(cudaMemcpy(alpha_body, D.alpha_b, sizeof(double) * D.nbody, cudaMemcpyDeviceToHost));
    if (passes_body) *passes_body = s->hv->S.ccd_passes_b;
    return IPC_OK;
}

// reads n 16-byte words (to fill L2 with clean lines of another buffer)
__global__ void k_touch(const uint4* __restrict__ p, size_t n, unsigned* sink) {
    unsigned acc = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint4 v = p[i];
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    if (acc == 0x9e3779b9u) *sink = acc;
}

// Replay of one stage's kernels on the scene's current state. The event pair
// on this system resolves about 2 us, coarse against kernels of 10-200 us,
// so two loops are timed whole: reps x (flush, preparation, stage) and reps x
// (flush, preparation); the stage's mean device time is their difference
// over reps (the flush evicts L2 before every launch in both).
template <class R>
int replay_impl(ipc_scene* s, int stage, int reps, void* flush, size_t flush_bytes, cudaStream_t st, double* ms) {
    Dev<R>& D = dev_of<R>(s);
    if (stage == 0 && !s->mas_built) return fail(IPC_ERR_INVALID, "replay: no blocks have been assembled yet");
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            for (auto& f : ev)
                if (f) cudaEventDestroy(f);
            return fail(IPC_ERR_CUDA, "cudaEventCreate failed");
        }
    KL(k_reset_flags<R><<<1, 1, 0, st>>>(D));
    if (stage == 4) launch_classify(D, D.C, st);  // the Woodbury lists of the current contacts, untimed
    auto one = [&](bool with_stage) {
        if (flush && flush_bytes >= 16)
            KL(k_touch<<<1184, 256, 0, st>>>(static_cast<const uint4*>(flush), flush_bytes / 16,
                                             static_cast<unsigned*>(flush)));
        if (stage == 3) launch_forms_prep(D, false, st);
        if (!with_stage) return;
        if (stage == 0)
            launch_invert(D, st);
        else if (stage == 2 || stage == 4)
            launch_blocks(D, D.g, D.z, D.C, stage == 4, st);
        else
            launch_forms_main(D, D.C, false, st);
    };
    one(true);  // warm the launch path
    cudaEventRecord(ev[0], st);
    for (int i = 0; i < reps; ++i) one(true);
    cudaEventRecord(ev[1], st);
    cudaEventRecord(ev[2], st);
    for (int i = 0; i < reps; ++i) one(false);
    cudaEventRecord(ev[3], st);
    float t1 = 0.f, t0 = 0.f;
    int rc = IPC_OK;
    if (cudaEventSynchronize(ev[3]) != cudaSuccess || cudaEventElapsedTime(&t1, ev[0], ev[1]) != cudaSuccess ||
        cudaEventElapsedTime(&t0, ev[2], ev[3]) != cudaSuccess)
        rc = fail(IPC_ERR_CUDA, std::string("replay: ") + cudaGetErrorString(cudaGetLastError()));
    for (auto& e : ev) cudaEventDestroy(e);
    if (rc != IPC_OK) return rc;
    CUDA_TRY(cudaMemcpy(&s->hv->S.async_timeout, &D.S->async_timeout, sizeof(int), cudaMemcpyDeviceToHost));
    if (s->hv->S.async_timeout) return fail(IPC_ERR_TIMEOUT, "replay: a bulk copy into shared memory did not complete");
    *ms = std::max(0.0, (double)(t1 - t0) / reps);
    return IPC_OK;
}

// ---- allocation-free preconditioner apply (no counterpart in the paper)
//
// For callers that must not allocate device memory while they run: a solver
// loop that shares the device with other busy streams, where cudaMalloc /
// cudaFree can synchronise the whole device, and processes whose device
// memory is owned by another allocator (a framework's caching pool), where
// one more allocation can fail. The MAS apply (Sec. 3.3, additive over
// levels) needs scratch only for the restricted residuals r_l and coarse
// solutions y_l of levels l >= 1, plus a status record for its bulk-copy
// waits; here they live in one static device array per device instead of
// the scene's arena, so the call writes nothing of the scene. The status
// record is cleared at the start of every call; every coarse residual and
// every coarse solution is written before it is read. Calls that overlap in
// time on one device (any scene, any stream) share this array and race.
constexpr size_t kNoAllocScratchBytes = 256 * 1024;
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
std::atomic<void*> g_noalloc_addr[kNoAllocMaxDevices];

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

bool device_array_on(const void* p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

template <class R>
int precond_noalloc_impl(ipc_scene* s, const void* g_dev, void* z_dev, cudaStream_t st) {
    const Dev<R>& D = dev_of<R>(s);
    if (!s->mas_built)
        return fail(IPC_ERR_INVALID,
                    "ipc_precond_apply_noalloc: the scene has no preconditioner yet (no RebuildMAS has run: call "
                    "ipc_step, ipc_eval_precond or ipc_eval_forms first)");
    int dev = -1;
    CUDA_TRY(cudaGetDevice(&dev));
    if (!device_array_on(D.blocks, dev))
        return fail(IPC_ERR_INVALID, "ipc_precond_apply_noalloc: the current device is not the scene's device");
    if (!device_array_on(g_dev, dev) || !device_array_on(z_dev, dev))
        return fail(IPC_ERR_INVALID, "ipc_precond_apply_noalloc: g and z must be device arrays on the scene's device");
    const size_t bytes = sizeof(R) * 3 * (size_t)D.nv;
    const char* gb = static_cast<const char*>(g_dev);
    const char* zb = static_cast<const char*>(z_dev);
    if (gb < zb + bytes && zb < gb + bytes) return fail(IPC_ERR_INVALID, "ipc_precond_apply_noalloc: g and z overlap");
    const size_t n_coarse = (size_t)D.coarse_off[D.nlev];
    const size_t status = align256(sizeof(Scalars));
    const size_t need = status + 2 * align256(sizeof(R) * n_coarse);
    if (need > kNoAllocScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "ipc_precond_apply_noalloc: the coarse levels need %zu bytes of scratch, above the %zu-byte "
                 "static limit; use ipc_eval_precond",
                 need, kNoAllocScratchBytes);
        return fail(IPC_ERR_CAPACITY, msg);
    }
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(IPC_ERR_INVALID, "ipc_precond_apply_noalloc: device ordinal above 63");
    void* base = g_noalloc_addr[dev].load(std::memory_order_acquire);
    if (!base) {
        // first call on this device: resolve the array's address (the
        // current device is the scene's, checked above)
        CUDA_TRY(cudaGetSymbolAddress(&base, g_noalloc_scratch));
        g_noalloc_addr[dev].store(base, std::memory_order_release);
    }
    unsigned char* b = static_cast<unsigned char*>(base);
    Dev<R> E = D;
    E.S = reinterpret_cast<Scalars*>(b);
    E.coarse_r = reinterpret_cast<R*>(b + status);
    E.coarse_y = reinterpret_cast<R*>(b + status + align256(sizeof(R) * n_coarse));
    CUDA_TRY(cudaMemsetAsync(E.S, 0, sizeof(Scalars), st));
    launch_precond(E, static_cast<const R*>(g_dev), static_cast<R*>(z_dev), E.C, false, st);
    CUDA_TRY(cudaGetLastError());
    // the bounded bulk-copy waits report through the status record: read it
    // (into host stack memory) once the apply has finished
    int timed_out = 0;
    CUDA_TRY(cudaMemcpyAsync(&timed_out, &E.S->async_timeout, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (timed_out)
        return fail(IPC_ERR_TIMEOUT, "ipc_precond_apply_noalloc: a bulk copy into shared memory did not complete; z is "
                                     "not defined");
    return IPC_OK;
}

ipc_scene* checked(ipc_scene* s) {
    if (!s) g_err = "null scene";
    return s;
}

}  // namespace

extern "C" {

void ipc_default_params(ipc_params* p) {
    memset(p, 0, sizeof *p);
    p->h = 1.0 / 30.0;
    p->dhat = 1e-3;
    p->kappa = 1.0;
    p->tol = 1e-3;
    p->delta = 0.3;
    p->eps_rot_deg = 25.0;
    p->ccd_shrink = 0.1;
    p->eps_sing = 1e-12;
    p->eps_abs = 1e-300;
    p->K = 8;
    p->iter_max = 10000;
    p->levels_max = 6;
    p->ls_max = 20;
    p->precision = IPC_PREC_FP64;
    p->contact_capacity = 0;
    p->broad_phase = 0;
    p->mas_mode = 0;
    p->ccd_mode = 0;
    p->graphs = 1;
    p->fp32_pivot_floor = 1e-6;
    p->grid_pair_capacity = 0;
    p->wait_polls = 1 << 22;
    p->apply_ctas = 0;
}

const char* ipc_last_error(void) { return g_err.c_str(); }

int ipc_scene_create(const ipc_scene_desc* desc, const ipc_params* params, const ipc_alloc_fns* alloc, ipc_scene** out) {
    if (!out || !desc || !params) return fail(IPC_ERR_INVALID, "null argument");
    *out = nullptr;
    if (!(params->h > 0) || !(params->dhat > 0) || !(params->kappa > 0) || params->K < 0 || params->K > kMaxK ||
        params->iter_max <= 0 || params->levels_max < 1 || params->ls_max < 0 || params->mas_mode < 0 ||
        params->mas_mode > 3 || params->ccd_mode < 0 || params->ccd_mode > 1 || params->apply_ctas < 0 ||
        params->apply_ctas > 16 ||
        (params->precision != IPC_PREC_FP64 && params->precision != IPC_PREC_FP32 &&
         params->precision != IPC_PREC_BF16_MAS) ||
        params->broad_phase < 0 ||
        params->broad_phase > 2)
        return fail(IPC_ERR_INVALID, "invalid parameters");
    ipc_scene* s = new ipc_scene();
    s->prm = *params;
    s->prec = params->precision;
    if (alloc) s->arena.fns = *alloc;
    std::string err;
    int r = build_host_mesh(desc, params->levels_max, &s->hm, &err);
    if (r != IPC_OK) {
        delete s;
        return fail(r, err);
    }
    if (cudaMallocHost(&s->hv, sizeof(HostView)) != cudaSuccess) {
        delete s;
        return fail(IPC_ERR_OOM, "pinned host allocation failed");
    }
    r = s->prec == IPC_PREC_FP64 ? setup_dev<double>(s) : setup_dev<float>(s);
    if (r != 0) {
        std::string msg = g_err;
        ipc_scene_destroy(s);
        return fail(r, msg);
    }
    // initial state must be separated: every active contact has d > 0
    int nc = 0;
    std::vector<double> x0 = s->hm.x0;
    r = s->prec == IPC_PREC_FP64
            ? eval_contacts_impl<double>(s, x0.data(), 0, &nc, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0)
            : eval_contacts_impl<float>(s, x0.data(), 0, &nc, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0);
    if (r != 0) {
        std::string msg = g_err;
        ipc_scene_destroy(s);
        return fail(r, msg);
    }
    if (s->hv->S.nonpos) {
        ipc_scene_destroy(s);
        return fail(IPC_ERR_INTERSECTING, "initial state has a contact at distance <= 0");
    }
    *out = s;
    return IPC_OK;
}

void ipc_scene_destroy(ipc_scene* s) {
    if (!s) return;
    // the scene's own stream and the legacy one; work the caller queued for
    // the scene on its streams must be complete (no device-wide wait: other
    // threads may be capturing graphs of other scenes)
    if (s->own) cudaStreamSynchronize(s->own);
    cudaStreamSynchronize(cudaStreamLegacy);
    s->arena.release();
    if (s->hv) cudaFreeHost(s->hv);
    delete s;
}

int ipc_step(ipc_scene* s, int n_steps, void* stream, ipc_step_stats* stats) {
    if (!checked(s)) return IPC_ERR_INVALID;
    if (n_steps < 0) return fail(IPC_ERR_INVALID, "negative step count");
    cudaStream_t st = (cudaStream_t)stream;
    return s->prec == IPC_PREC_FP64 ? step_impl<double>(s, n_steps, st, stats) : step_impl<float>(s, n_steps, st, stats);
}

int ipc_set_state(ipc_scene* s, const double* x, const double* v, int on_device, void* stream) {
    if (!checked(s) || !x) return fail(IPC_ERR_INVALID, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    size_t n3 = 3 * (size_t)s->hm.nv;
    double* dx = s->prec == IPC_PREC_FP64 ? s->dd.x : s->df.x;
    double* dv = s->prec == IPC_PREC_FP64 ? s->dd.v : s->df.v;
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // a non-finite coordinate is refused before it reaches the scene: no
    // kernel ever sees one from the caller
    unsigned long long bad = 0;
    if (on_device) {
        CUDA_TRY(cudaMemsetAsync(s->nonfinite, 0, sizeof(unsigned long long), st));
        KL(k_count_nonfinite<double><<<64, 256, 0, st>>>(x, n3, s->nonfinite));
        if (v) KL(k_count_nonfinite<double><<<64, 256, 0, st>>>(v, n3, s->nonfinite));
        CUDA_TRY(cudaMemcpyAsync(&s->hv->nonfinite, s->nonfinite, sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        bad = s->hv->nonfinite;
    } else {
        for (size_t i = 0; i < n3; ++i) bad += !std::isfinite(x[i]) + (v ? !std::isfinite(v[i]) : 0);
    }
    if (bad) return fail(IPC_ERR_INVALID, "non-finite position or velocity (state unchanged)");
    CUDA_TRY(cudaMemcpyAsync(dx, x, sizeof(double) * n3, kind, st));
    s->cand_ok = false;
    if (v)
        CUDA_TRY(cudaMemcpyAsync(dv, v, sizeof(double) * n3, kind, st));
    else
        CUDA_TRY(cudaMemsetAsync(dv, 0, sizeof(double) * n3, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return IPC_OK;
}

int ipc_query(ipc_scene* s, int what, void* dst, size_t bytes, void* stream) {
    if (!checked(s) || !dst) return fail(IPC_ERR_INVALID, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    size_t n3 = 3 * (size_t)s->hm.nv;
    bool f64 = s->prec == IPC_PREC_FP64;
    auto need = [&](size_t n) { return bytes >= n; };
    switch (what) {
        case IPC_Q_POSITIONS:
        case IPC_Q_VELOCITIES: {
            if (!need(sizeof(double) * n3)) return fail(IPC_ERR_INVALID, "destination too small");
            const double* src = what == IPC_Q_POSITIONS ? (f64 ? s->dd.x : s->df.x) : (f64 ? s->dd.v : s->df.v);
            CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(double) * n3, cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            return IPC_OK;
        }
        case IPC_Q_N_VERTS:
            if (!need(sizeof(int))) return fail(IPC_ERR_INVALID, "destination too small");
            *(int*)dst = s->hm.nv;
            return IPC_OK;
        case IPC_Q_N_CONTACTS: {
            if (!need(sizeof(int))) return fail(IPC_ERR_INVALID, "destination too small");
            std::vector<double> x(n3);
            CUDA_TRY(cudaMemcpy(x.data(), f64 ? s->dd.x : s->df.x, sizeof(double) * n3, cudaMemcpyDeviceToHost));
            int n = 0;
            int r = f64 ? eval_contacts_impl<double>(s, x.data(), 0, &n, 0, 0, 0, 0, 0, 0, st)
                        : eval_contacts_impl<float>(s, x.data(), 0, &n, 0, 0, 0, 0, 0, 0, st);
            if (r) return r;
            *(int*)dst = n;
            return IPC_OK;
        }
        case IPC_Q_SUBDOMAIN_ALPHA: {
            size_t ng = s->hm.ngroups[0];
            if (!need(sizeof(double) * ng)) return fail(IPC_ERR_INVALID, "destination too small");
            CUDA_TRY(cudaMemcpy(dst, f64 ? s->dd.alpha : s->df.alpha, sizeof(double) * ng, cudaMemcpyDeviceToHost));
            return IPC_OK;
        }
        case IPC_Q_N_SUBDOMAINS:
            if (!need(sizeof(int))) return fail(IPC_ERR_INVALID, "destination too small");
            *(int*)dst = s->hm.ngroups[0];
            return IPC_OK;
        case IPC_Q_TRACE_LEN:
            if (!need(sizeof(int))) return fail(IPC_ERR_INVALID, "destination too small");
            *(int*)dst = (int)s->trace.size();
            return IPC_OK;
        case IPC_Q_TRACE: {
            size_t n = std::min(s->trace.size(), bytes / sizeof(ipc_iter_record));
            memcpy(dst, s->trace.data(), n * sizeof(ipc_iter_record));
            return IPC_OK;
        }
        case IPC_Q_SURFACE_COUNTS: {
            if (!need(3 * sizeof(int))) return fail(IPC_ERR_INVALID, "destination too small");
            int* o = (int*)dst;
            o[0] = (int)s->hm.sv.size();
            o[1] = (int)(s->hm.sf.size() / 3);
            o[2] = (int)(s->hm.se.size() / 2);
            return IPC_OK;
        }
        case IPC_Q_N_BODIES:
            if (!need(sizeof(int))) return fail(IPC_ERR_INVALID, "destination too small");
            *(int*)dst = s->hm.nbody;
            return IPC_OK;
        case IPC_Q_FP64_BLOCKS: {
            if (!need(sizeof(int))) return fail(IPC_ERR_INVALID, "destination too small");
            const int nb = f64 ? s->dd.blk_off[s->dd.nlev] : s->df.blk_off[s->df.nlev];
            if (f64) {
                *(int*)dst = nb;
                return IPC_OK;
            }
            std::vector<int> fl(std::max(nb, 1));
            CUDA_TRY(cudaMemcpyAsync(fl.data(), s->df.invflag, sizeof(int) * nb, cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            int n = 0;
            for (int i = 0; i < nb; ++i) n += fl[i] != 0;
            *(int*)dst = n;
            return IPC_OK;
        }
        case IPC_Q_PIVOT_FIXES: {
            if (!need(sizeof(int))) return fail(IPC_ERR_INVALID, "destination too small");
            CUDA_TRY(cudaMemcpyAsync(dst, f64 ? s->dd.pivfix : s->df.pivfix, sizeof(int), cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            return IPC_OK;
        }
        case IPC_Q_APPLY_CTAS:
            if (!need(sizeof(int))) return fail(IPC_ERR_INVALID, "destination too small");
            *(int*)dst = f64 ? s->dd.apply_ctas : s->df.apply_ctas;
            return IPC_OK;
        case IPC_Q_BBOX_DIAG:
            if (!need(sizeof(double))) return fail(IPC_ERR_INVALID, "destination too small");
            *(double*)dst = s->hm.bbox_diag;
            return IPC_OK;
        default:
            return fail(IPC_ERR_INVALID, "unknown query kind");
    }
}

int ipc_query_level(ipc_scene* s, int level, int* n_nodes, int* n_groups, int* group_of_node, int* slot_of_node) {
    if (!checked(s)) return IPC_ERR_INVALID;
    if (level < 0 || level >= s->hm.nlev) return fail(IPC_ERR_INVALID, "level out of range");
    if (n_nodes) *n_nodes = s->hm.nnodes[level];
    if (n_groups) *n_groups = s->hm.ngroups[level];
    if (group_of_node) memcpy(group_of_node, s->hm.group_of[level].data(), sizeof(int) * s->hm.nnodes[level]);
    if (slot_of_node) memcpy(slot_of_node, s->hm.slot_of[level].data(), sizeof(int) * s->hm.nnodes[level]);
    return s->hm.nlev;
}

int ipc_query_surface(ipc_scene* s, int* verts, int* tris, int* edges) {
    if (!checked(s)) return IPC_ERR_INVALID;
    if (verts) memcpy(verts, s->hm.sv.data(), sizeof(int) * s->hm.sv.size());
    if (tris) memcpy(tris, s->hm.sf.data(), sizeof(int) * s->hm.sf.size());
    if (edges) memcpy(edges, s->hm.se.data(), sizeof(int) * s->hm.se.size());
    return IPC_OK;
}

long long ipc_kernel_launches(void) { return g_kernel_launches.load(); }

int ipc_profile_enable(ipc_scene* s, int enable) {
    if (!checked(s)) return IPC_ERR_INVALID;
    for (auto& q : s->prof.pending) cudaEventSynchronize(q.b);
    s->prof.resolve();
    s->prof.on = enable != 0;
    if (enable) {
        for (int i = 0; i < 8; ++i) {
            s->prof.ms[i] = 0.0;
            s->prof.n[i] = 0;
        }
    }
    return IPC_OK;
}

int ipc_profile_read(ipc_scene* s, ipc_profile* out) {
    if (!checked(s) || !out) return IPC_ERR_INVALID;
    for (auto& q : s->prof.pending) cudaEventSynchronize(q.b);
    s->prof.resolve();
    for (int i = 0; i < 8; ++i) {
        out->ms[i] = s->prof.ms[i];
        out->launches[i] = s->prof.n[i];
    }
    return IPC_OK;
}

int ipc_eval_energy_grad(ipc_scene* s, const double* x, const double* xtilde, double* energy, double* g, void* stream) {
    if (!checked(s) || !x || !xtilde) return fail(IPC_ERR_INVALID, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    return s->prec == IPC_PREC_FP64 ? eval_energy_impl<double>(s, x, xtilde, energy, g, st)
                                    : eval_energy_impl<float>(s, x, xtilde, energy, g, st);
}

int ipc_eval_contacts(ipc_scene* s, const double* x, int cap, int* n, int* type, int* ids, int* verts, double* dist,
                      double* k, double* grad12, void* stream) {
    if (!checked(s) || !x) return fail(IPC_ERR_INVALID, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    return s->prec == IPC_PREC_FP64 ? eval_contacts_impl<double>(s, x, cap, n, type, ids, verts, dist, k, grad12, st)
                                    : eval_contacts_impl<float>(s, x, cap, n, type, ids, verts, dist, k, grad12, st);
}

int ipc_eval_precond(ipc_scene* s, const double* x_base, const double* x_curr, const double* g, double* z, void* stream) {
    if (!checked(s) || !x_base || !g || !z) return fail(IPC_ERR_INVALID, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    return s->prec == IPC_PREC_FP64 ? eval_precond_impl<double>(s, x_base, x_curr, g, z, st)
                                    : eval_precond_impl<float>(s, x_base, x_curr, g, z, st);
}

int ipc_eval_forms(ipc_scene* s, const double* x_base, const double* x_curr, const double* z, const double* p,
                   double out[3], void* stream) {
    if (!checked(s) || !x_base || !z || !p || !out) return fail(IPC_ERR_INVALID, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    return s->prec == IPC_PREC_FP64 ? eval_forms_impl<double>(s, x_base, x_curr, z, p, out, st)
                                    : eval_forms_impl<float>(s, x_base, x_curr, z, p, out, st);
}

int ipc_profile_replay(ipc_scene* s, int stage, int reps, void* flush, size_t flush_bytes, void* stream,
                       double* ms_mean) {
    if (!checked(s) || !ms_mean) return fail(IPC_ERR_INVALID, "null argument");
    if ((stage != 0 && stage != 2 && stage != 3 && stage != 4) || reps < 1)
        return fail(IPC_ERR_INVALID, "replay: stage must be 0, 2, 3 or 4, reps >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    return s->prec == IPC_PREC_FP64 ? replay_impl<double>(s, stage, reps, flush, flush_bytes, st, ms_mean)
                                    : replay_impl<float>(s, stage, reps, flush, flush_bytes, st, ms_mean);
}

int ipc_profile_fma_peak(int precision, double target_ms, double* tflops) {
    if (!tflops || !(target_ms > 0.0) || target_ms > 1000.0 ||
        (precision != IPC_PREC_FP64 && precision != IPC_PREC_FP32))
        return fail(IPC_ERR_INVALID, "fma peak: precision FP64 or FP32, 0 < target_ms <= 1000");
    const int r = precision == IPC_PREC_FP64 ? measure_fma_peak<double>(target_ms, tflops)
                                             : measure_fma_peak<float>(target_ms, tflops);
    return r == 0 ? IPC_OK : fail(IPC_ERR_CUDA, "fma peak: CUDA error");
}

int ipc_precond_apply_noalloc(ipc_scene* s, const void* g_dev, void* z_dev, void* stream) {
    if (!checked(s) || !g_dev || !z_dev) return fail(IPC_ERR_INVALID, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    return s->prec == IPC_PREC_FP64 ? precond_noalloc_impl<double>(s, g_dev, z_dev, st)
                                    : precond_noalloc_impl<float>(s, g_dev, z_dev, st);
}

int ipc_eval_ccd(ipc_scene* s, const double* x, const double* p, double* alpha, int* passes, double* alpha_body,
                 int* passes_body, void* stream) {
    if (!checked(s) || !x || !p || !alpha) return fail(IPC_ERR_INVALID, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    return s->prec == IPC_PREC_FP64 ? eval_ccd_impl<double>(s, x, p, alpha, passes, alpha_body, passes_body, st)
                                    : eval_ccd_impl<float>(s, x, p, alpha, passes, alpha_body, passes_body, st);
}

}  // extern "C"
