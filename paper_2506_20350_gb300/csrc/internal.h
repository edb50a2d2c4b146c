// Host-side plan object and the internal launch interface shared by the
// translation units of libbttb.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "bttb.h"
#include "check.cuh"

namespace bttb {

constexpr int kMaxRadixStages = 24;
constexpr int kMaxM = 2048;          // largest FFT length (grid side) supported
constexpr int kContractKC = 4;       // right-hand sides per pass of the block product

// Radix plan and twiddle tables of one FFT length.  Tables hold
// exp(-2 pi i t / M) for t < M, followed by five real constants of the
// radix-3/5 butterflies in the real parts: cos(2pi/5), cos(4pi/5),
// sin(2pi/5), sin(4pi/5), sin(pi/3).
struct FftPlan {
    int M = 0;
    int nst = 0;
    int radix[kMaxRadixStages] = {};
    double2 *tw_f64 = nullptr;   // device
    float4 *tw_df = nullptr;     // device, double-float {re.hi, im.hi, re.lo, im.lo}
    float2 *tw_f32 = nullptr;    // device
};

// One batched strided 1-D FFT pass (see fft.cu).
struct FftPass {
    const void *in;
    void *out;
    long in_cs, in_os, in_ns;     // strides (elements) of column, outer index, element index
    long out_cs, out_os, out_ns;
    const int *in_sel;            // optional device index: input offset += (*in_sel) * in_sel_stride
    long in_sel_stride;
    const double *in_scale;       // optional device per-column scale applied on load (binary64)
    const int *active;            // optional device per-column flags: inactive columns are skipped
    int O;                        // number of outer indices
    int pdim;                     // contiguous inner count (bases, or b*b entries)
    int ncols;
    int nin, nout;                // nonzero input elements, kept output elements
    int M, nst;
    int radix[kMaxRadixStages];
    unsigned nsmagic[kMaxRadixStages];   // ceil(2^32 / Ns) of each stage (Ns = product of the earlier radices)
    const void *tw;
    int P, log2P;                 // inner chunk per CTA (power of two)
    int cpb;                      // columns per CTA (> 1: the next column's input is prefetched while one runs)
};

enum Prec { PREC_DF64 = BTTB_MV_FP64, PREC_F32 = BTTB_MV_FP32, PREC_F64N = BTTB_MV_FP64_NATIVE,
            PREC_TC = BTTB_MV_TC_3XTF32, PREC_TCB = BTTB_MV_TC_BF16X3 };
// Columns from which BTTB_MV_TC_3XTF32 runs the block product on the tensor cores.
constexpr int kTcMinCols = 16;
// FFT passes and vector format of a product precision (the tensor-core product is binary32 around the GEMM).
inline bool is_tc_prec(int prec) { return prec == PREC_TC || prec == PREC_TCB; }
inline int fft_prec_of(int prec) { return is_tc_prec(prec) ? PREC_F32 : prec; }

struct GmresWork;
struct Learned;

// Launch shape of the fused y-level transform + block product (ycontract.cu) for one precision and column
// count: cluster size, shares, ring, shared-memory offsets.  ok < 0: not decided yet, 0: does not fit.
struct YcShape {
    int ok = -1;
    int Q = 0, pshare = 0, kshare = 0, Qc = 0, nchunks = 0, nstages = 0, nfix = 0;
    unsigned stage_bytes = 0, off_g1 = 0, off_tw = 0, off_f0 = 0, off_f1 = 0, off_uh = 0, off_ring = 0;
    size_t smem = 0;
};

// Forms of a product of one to four columns (bttb_plan_debug BTTB_DEBUG_PRODUCT_ROUTE).
enum ProductRoute { ROUTE_AUTO = 0, ROUTE_PASSES = 1, ROUTE_FUSED_FFT2 = 2, ROUTE_FUSED_Y = 3, ROUTE_PERSISTENT = 4 };

struct Plan {
    int nx = 0, ny = 0, b = 0, mx = 0, my = 0, max_rhs = 0;
    long n = 0;                   // nx*ny*b
    long bins = 0;                // mx*my
    unsigned prec_mask = 0;
    cudaStream_t stream = nullptr;
    int dev = 0, nsm = 0;
    size_t smem_optin = 0;
    FftPlan fx, fy;
    int fft_pmax = 16;            // widest batch chunk of an FFT pass (power of two; autotuned in batches)
    bool in_batch = false;        // runs beside other plans' kernels (bttb_batch): prefer occupancy

    // Spectrum copies, scaled by 1/(mx*my).  Bin k holds its b x b block
    // column-major (entry (p, q) at q*b + p) at offset k*gbs elements.
    float2 *ghat_hi = nullptr;    // binary32 rounding of the spectrum
    float2 *ghat_lo = nullptr;    // binary32 remainder (double-float low plane)
    double2 *ghat_f64 = nullptr;  // binary64 copy
    long gbs = 0;
    bool have_gen = false;

    // Block-Jacobi: R_0^{-1} (column-major, rows padded to a multiple of 4, binary32) for P_K of Sec. III-B.
    float2 *bj_inv = nullptr;
    bool bj_ready = false;

    // Product workspace: two buffers of bins * ubs * 16 bytes.
    void *wsA = nullptr, *wsB = nullptr;
    long ubs = 0;                 // bin stride (elements) of the spectral vectors
    size_t ws_bytes = 0;

    // Failure-path test hooks (bttb_plan_debug): bound of the kernels' pipeline waits, and the number of
    // coming uncaptured one-to-eight-column block products that withhold one mbarrier arrival.
    unsigned long long wait_ns = 2000000000ull;
    int withhold = 0;
    int route_f32 = ROUTE_AUTO;   // form of the few-column binary32 / tensor-core product (autotuned or forced)
    int route_df = ROUTE_AUTO;    // form of the few-column double-float / binary64 product
    YcShape yc[2][4];             // fused y-level product shapes: [binary32, double-float][columns - 1]
    int yc_force_q = 0;           // cluster size of the fused y-level product (0: the largest resident one)

    GmresWork *gw = nullptr;
    Learned *learned = nullptr;   // attached learned preconditioner (learned.cu), not owned
    int *d_err = nullptr;         // device error word (first word of a 64-byte block)
    unsigned long long *d_gbar = nullptr;   // grid-barrier arrival counter of the whole-product kernel (d_err + 16 B)
    size_t bytes_held = 0;

    // Profiling (bttb_profile): event pairs around timed launches, launch count.
    struct ProfRec { int ev0, ev1, kid; double bytes; };
    int prof = 0;                 // 0 off, 1 block product + FFT (outside graphs), 2 every timed kernel
    std::vector<cudaEvent_t> ev_pool;
    int ev_used = 0;
    std::vector<ProfRec> recs;
    long launches = 0;
    // While a graph is captured, timed launches get their own events, tagged
    // with the Arnoldi step; accumulated after each replay into acc_*.
    struct GraphRec { cudaEvent_t e0, e1; int kid; double bytes; int step; };
    std::vector<GraphRec> *sink = nullptr;
    int sink_step = 0;
    static constexpr int kMaxKid = 32;
    double acc_ms[kMaxKid] = {}, acc_bytes[kMaxKid] = {};
    long acc_n[kMaxKid] = {};
};

// Profiling helpers (bttb.cu).  prof_begin returns a token for prof_end, or -1.
int prof_begin(Plan *p, int kid);
void prof_end(Plan *p, int token, double bytes);
inline void count_launch(Plan *p, int n = 1) { p->launches += n; }

// Launch with the programmatic-stream-serialisation attribute: the kernel may be
// scheduled while its predecessor drains; it waits on griddepcontrol.wait.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Thread-local error message helpers (bttb.cu).
int set_error(Plan *p, int code, const std::string &msg);
int check_cuda(Plan *p, cudaError_t e, const char *what);

// fft.cu
int fft_plan_init(Plan *p, FftPlan &f, int M);
void fft_plan_free(FftPlan &f);
int fft_pass_launch(Plan *p, FftPass a, int prec, int infmt, int outfmt, bool inverse);
// Radix plan, batch chunk P (at most pmax) and twiddles of a pass, without launching it (a.cpb = 0: choose).
int fft_pass_prepare(Plan *p, FftPass &a, int prec, int pmax);
// Both FFT levels of a product in one kernel (few columns): forward cell-ordered x (cellfmt) -> u^, or
// inverse v^ -> cell-ordered y (cellfmt); ld is the cell-ordered vector's column stride.
int fft2_fused_launch(Plan *p, const void *in, void *out, long ld, int ncols, int prec, int cellfmt, bool inverse,
                      const int *in_sel, long in_sel_stride, const double *in_scale, const int *active);
size_t fft2_fused_smem(const Plan *p, int prec);
// Products of at most this many columns run the fused FFT when its grid fits shared memory.
constexpr int kFusedFftMaxCols = 4;
int spectrum_compute(Plan *p, const void *gen, bttb_dtype dtype, int gen_is_host);
int smallest_5smooth(int n);

// tcgemm.cu: the many-column per-bin GEMM on the tcgen05 tensor cores (3xTF32, or split-BF16x3 with
// fmt_bf16); fits when b is even and at most 64 and k >= kTcMinCols.
bool tcgemm_fits(const Plan *p, int k);
int tcgemm_launch(Plan *p, int fmt_bf16, const void *u, void *v, int k);

// contract.cu
int contract_launch(Plan *p, int prec, const void *u, void *v, int k, const int *active = nullptr);

// contract.cu: the whole product (the four strided passes and the block product as phases of one
// persistent kernel); whether it takes k columns of this precision, and its launch (formats as matvec_run).
bool product_persistent_fits(Plan *p, int prec, int k);
int product_persistent_launch(Plan *p, const void *x, int xfmt, long ldx, void *y, int yfmt, long ldy, int k,
                              int prec, const int *in_sel, long in_sel_stride, const double *in_scale,
                              const int *active);

// ycontract.cu: whether the fused y-level transform + block product takes k columns in this precision
// (decided once per plan), and its launch on the x pass's output U ([c][iy][kx][p]) into V (same layout).
bool ycontract_fits(Plan *p, int prec, int k);
int ycontract_launch(Plan *p, int prec, const void *U, void *V, int k, const int *active);
int ycontract_probe(Plan *p, int prec, int k, int Q);

// matvec.cu
// y[:, c] = Z x[:, c]; xfmt/yfmt are VecFmt values; in_sel/in_scale as in FftPass.
int matvec_run(Plan *p, const void *x, int xfmt, long ldx, void *y, int yfmt, long ldy, int nrhs, int prec,
               const int *in_sel = nullptr, long in_sel_stride = 0, const double *in_scale = nullptr,
               const int *active = nullptr);
// ProductRoute a product of nrhs columns in precision prec takes.
int product_route(Plan *p, int nrhs, int prec);
int block_jacobi_run(Plan *p, const void *x, int xfmt, long ldx, void *z, int zfmt, long ldz, int nrhs,
                     const int *in_sel = nullptr, long in_sel_stride = 0, const int *active = nullptr);
int block_jacobi_setup(Plan *p, const double2 *t00_host);

// gmres.cu
int gmres_solve(Plan *p, const void *V, void *I, int nrhs, long ld, const bttb_gmres_opts *o,
                bttb_col_result *out);
void gmres_free(Plan *p);

// learned.cu: z = P_K^{-1} x + f(x) with the plan's attached learned correction.
int learned_apply_run(Plan *p, const void *x, int xfmt, long ldx, void *z, int zfmt, long ldz, int nc);
int learned_max_cols(const Learned *L);

}  // namespace bttb

// The opaque handle of the C ABI wraps a plan.
struct bttb_plan_s {
    bttb::Plan p;
};
