// engine.h -- state of one library context and the host-side steps of the
// two-site DMRG iteration (Sec. II.B of arXiv:2412.04676).
#pragma once

#include <cusolverDn.h>

#include <map>
#include <memory>
#include <tuple>
#include <vector>

#include "core.h"
#include "kernels.h"
#include "mpo.h"
#include "spill.h"
#include "tc.h"

namespace gbd {

// A site tensor of Eq. 2 in isometric form.
//  kind 0 (left): U_Q, rows = enlarged-left basis of bond k, cols = bond k+1 sector Q
//  kind 1 (right): V_Q, rows = enlarged-right basis of bond k+1 (labelled at
//  cut k), cols = bond k sector Q.
struct Iso {
    int kind = -1;
    EBasis basis;
    Bond out;
    std::vector<long long> off;  // per out sector, -1 if absent
    long long total = 0;
    DevBuf data;
    std::vector<double> host;    // host copy (imported or exported)
};

// Packed (serialised) copy of an environment in pinned host memory.
struct HostEnv {
    unsigned char* host = nullptr;   // packages (mapped pinned)
    size_t cap = 0, bytes = 0;
    bool valid = false;              // holds a complete save
    cudaEvent_t done = nullptr;      // last save into `host` finished
    int npk = 0;
    unsigned char* meta = nullptr;   // pack/unpack item + chunk tables (mapped pinned)
    size_t meta_cap = 0;
    unsigned long long* cks_dev = nullptr;   // per-package checksum accumulators
    unsigned long long* cks_host = nullptr;  // verification copy (pinned)
    size_t cks_cap = 0;
    bool pending = false;            // load enqueued, not yet verified
    cudaEvent_t loaded = nullptr;
    std::vector<unsigned long long> want;
    // bounded store (host_store_bytes): the packed stream may live in the spill file
    bool spilled = false;            // payload only in the spill file (host == nullptr)
    bool restoring = false;          // read back into `host` in flight (job)
    std::shared_ptr<SpillJob> job;   // spill write or restore read in flight
    long long file_off = -1;         // this id's region of the spill file
    size_t file_cap = 0;
    unsigned long long stamp = 0;    // last save or load, for the choice of spill victims
};

// Enlarged operators and product plans at one two-site position b.
struct Heff {
    int b = -1;
    EBasis bL, bR;
    std::vector<Q> sq;
    std::vector<int> sL, sR;
    std::vector<long long> soff;
    long long dim = 0;
    OpSet OL, OR;
    GemmPlan p1, p2;         // FP64 product plans (built at the first FP64 product)
    bool fp64_ready = false;
    struct Pair { int c, bl, br, s_out, s_in; long long xoff; };
    std::vector<Pair> pairs; // (class, left block, right block) with matching sectors
    long long xtot = 0;      // FP64 phase-1 output elements
    DevBuf X, xin, yout, diag;
    bool diag_ready = false;
    long long ngemm = 0;
    double flops = 0.0, op_bytes = 0.0, mixed_bytes = 0.0, mixed_x_bytes = 0.0;
    // device memory model (bytes): enlarged FP64 arenas, tensor-core operator
    // planes of each form, phase-1 intermediates
    double mem_ops = 0.0, mem_bf16x3 = 0.0, mem_sliced = 0.0, mem_x64 = 0.0, mem_xtc = 0.0;
    TcHeff tc;               // mixed-precision (BF16x3, tcgen05) operands and plans
    bool tc_ready = false;
    int sector_of(const Q& q) const {
        auto it = std::lower_bound(sq.begin(), sq.end(), q);
        if (it == sq.end() || *it != q) return -1;
        return int(it - sq.begin());
    }
};

// The links of one enlargement (side, cut) between input and output operator
// classes for each local matrix element, with their coefficients: copy-sum
// lists for sparse links, dense coefficient matrices for the others.  They
// depend only on the MPO (Eq. 1 split at the cut), so they are built once per
// context and integrals, and reused by every sweep.
struct EnlLink {
    int ci, co, s, t;
    std::vector<double> W;  // T_in x T_out (dense links)
    long long doff = 0;     // offset of W in `wall`
};
struct EnlLinks {
    bool built = false;
    std::vector<EnlLink> links;
    std::vector<char> sparse;
    std::map<std::tuple<int, int, int>, std::vector<int>> by_cst;  // (output class, s, t) -> links
    std::vector<double> wall;       // dense coefficient matrices, concatenated
    std::vector<int> link_col0;     // sparse link -> first CopyCol (output layer 0)
    std::vector<int> amax;          // sparse link -> largest input layer its copies read
    std::vector<CopyCol> ccols;
    std::vector<CopyCoef> ccoefs;
};

struct Ctx {
    gbd_config cfg{};
    bool have_ints = false, cuda_ready = false;
    int L = 0;
    std::vector<double> h, eri;
    double ecore = 0.0;
    Mpo mpo;
    std::vector<Bond> bonds;
    std::vector<Iso> sites;
    std::vector<std::vector<double>> site_blocks_data;
    std::vector<std::vector<int>> site_blocks_meta;
    std::vector<int> site_kind;
    std::vector<std::unique_ptr<OpSet>> envL, envR;
    std::vector<HostEnv> hostL, hostR;
    std::unique_ptr<SpillStore> spill;   // created at the first spill
    std::vector<EnlLinks> enl_links[2];  // per side and cut; cleared with the integrals
    size_t pinned_bytes = 0;             // packed-stream buffers of the host store
    unsigned long long io_stamp = 0;
    cudaStream_t cs = nullptr, ios = nullptr;
    cusolverDnHandle_t sol = nullptr;
    static constexpr int kEigStreams = 16;
    cudaStream_t eig_st[kEigStreams] = {nullptr};
    cusolverDnHandle_t eig_sol[kEigStreams] = {nullptr};
    DevBuf eig_work[kEigStreams];
    std::vector<char> eig_host[kEigStreams];   // host workspace of the batched eigensolver
    cusolverDnParams_t eig_params = nullptr;
    Heff H;
    DevBuf psi;
    bool psi_valid = false;
    int psi_b = -1;
    // scratch
    GemmPlan plan_a, plan_b, plan_c;
    DevBuf scratch_w, scratch_tmp, scratch_dot, scratch_small, scratch_items, scratch_srcs, scratch_cols, scratch_coefs;
    DevBuf env_sl_w, env_sl_e, env_err;  // sliced operands of the tensor-core enlargement
    DevBuf dav_V, dav_AV, dav_r, dav_t, dav_x, dav_ax, dav_tmp, dav_best;
    DevBuf stage;  // device staging for pack/unpack through pageable memory
    // statistics
    std::vector<double> step_energy;
    double io_d2h = 0, io_h2d = 0, io_exposed_ms = 0, pack_ms = 0, save_ms = 0;
    struct PendingSave { cudaEvent_t a, b; };
    std::vector<PendingSave> saves;   // timing events of asynchronous saves
    double ms_matvec_acc = 0;
    int matvec_count = 0;
    bool last_dav_quick = false;  // previous mixed Davidson met its tolerance at the first anchor
    TcTune last_tune;             // the autotuner's last finished choice (trials or cache hit)
    int last_tune_b = -1;         // its position
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // phase timers (ms): host planning and device execution
    enum { T_ENL_HOST, T_ENL_DEV, T_REN_HOST, T_REN_DEV, T_EIG, T_POLISH, T_TCPREP, T_DAV_HOST, T_ENL_GFLOP, T_REN_GFLOP, T_TC_ISSUE1, T_TC_ISSUE2,
           T_PROD_MS0, T_PROD_MS1, T_PROD_MS2, T_PROD_N0, T_PROD_N1, T_PROD_N2, T_TC_ISSUE_SL,
           T_PREP_SPLIT, T_PREP_PLAN, T_PREP_UPLOAD, T_PROD_GF0, T_PROD_GF1, T_PROD_GF2,
           T_REN_TC_GFLOP, T_ENL_TC_GFLOP,
           // device time of the phases of gbd_step on the compute stream (host gaps included)
           T_PH_RESIDENT, T_PH_ENLARGE, T_PH_DAVIDSON, T_PH_RHO_EIG, T_PH_RENORM, T_PH_NEXT, T_PH_IO,
           T_ENL_H_LINKS, T_ENL_H_SUBS, T_ENL_H_ITEMS, T_PROD_GB1, T_PROD_XGB1, T_PROD_MS_PB, T_PROD_N_PB, T_RECOMP_MS, T_RECOMP_N,
           T_SPILL_GB, T_RESTORE_GB, T_SPILL_WAIT_MS, T_PROD_MS_TP, T_PROD_N_TP, T_PROD_MS_FZ, T_PROD_N_FZ, T_COUNT };
    std::vector<std::pair<int, cudaEvent_t>> marks;  // phase boundaries of the running step
    std::vector<cudaEvent_t> mark_pool;
    double timers[T_COUNT] = {0};
};

void ensure_cuda(Ctx& C);
void destroy_ctx(Ctx& C);
void load_integrals(Ctx& C, int L, const double* h, const double* eri, double ecore);
void import_site(Ctx& C, int k, int kind, int nblk, const int* meta, const double* data);
void finalize_sites(Ctx& C);
void build_envs(Ctx& C, int b);
void setup_heff(Ctx& C, int b);
void export_site(Ctx& C, int k, int* kind, std::vector<int>& meta, std::vector<double>& data);
double wall_ms();  // host wall clock in ms
void step_mark(Ctx& C, int phase);  // phase (a T_PH_* index) starts now on the compute stream
void step_marks_flush(Ctx& C);      // after the stream is synchronised: accumulate the phase times
void apply_heff_dev(Ctx& C, const double* in, double* out, int precision);
void heff_diag(Ctx& C);
int davidson(Ctx& C, double* psi_host, double* energy, gbd_dav_stats* st);
double truncate_step(Ctx& C, int dir, int Dmax);
int sweep(Ctx& C, int nsweeps, int D, gbd_sweep_stats* st);
int run_step(Ctx& C, int b, int dir, int D, gbd_step_stats* st);  // GBD_OK or GBD_WARN_NOT_CONVERGED
void collect_saves(Ctx& C, bool wait);
void make_resident(Ctx& C, int side, int cut);  // loads an offloaded environment back (checksums verified)
void offload_env(Ctx& C, int side, int cut);    // asynchronous save to pinned host memory, then device release
bool env_checkpoint(const Ctx& C, int side, int cut);  // saved to the host store (env_recompute)
void rebuild_env(Ctx& C, int side, int cut);   // recomputation from the nearest stored environment

// pack / unpack (serialisation)
size_t pack_size(const OpSet& E);
void pack_env(Ctx& C, const OpSet& E, unsigned char* dst, bool dst_device_or_pinned, cudaStream_t st);
void unpack_env(Ctx& C, OpSet& E, const unsigned char* src, size_t bytes, bool src_device_or_pinned, cudaStream_t st);
OpSet* env_of(Ctx& C, int side, int cut, bool create);

// thread-local message returned by gbd_last_error()
void set_last_error(const char* msg);

}  // namespace gbd
