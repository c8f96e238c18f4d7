// ctx.h -- host-side state of a GLD context and of a batch of contexts,
// shared by the translation units of the C ABI (api.cu, serve.cu).
#pragma once

#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "gld.h"
#include "launch.h"

using namespace gld;

struct gld_ctx {
    gld_params prm{};
    StepParams P{};
    int device = 0, num_sms = 0;
    cudaStream_t st = nullptr;   // the caller's stream
    cudaStream_t cap = nullptr;  // private stream used only to capture graphs
    cudaStream_t cap2 = nullptr; // fills the bodies of conditional graph nodes
    cudaStream_t cap3 = nullptr; // the overlapped next-step convolution of the graph
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool overlap_graph = false;  // the graph computes each step's successor convolution
    long long conv_valid_step = -1;  // the step whose projections `conv` already holds
    std::vector<void*> allocs;
    std::vector<size_t> alloc_sizes;
    size_t bytes = 0;  // device bytes held
    ParticleBuffers B{};
    float* W = nullptr;
    CUtensorMap wmap{};      // W in split form as 32 x 64 FP16 boxes for the tensor-core filter
    bool have_wmap = false;  // stepped alone, the ring holds the split form (P.wsplit)
    float* Acp = nullptr;
    int la = 0;
    float* coef = nullptr;
    float* g0 = nullptr;
    float* ftab = nullptr;
    float* fptab = nullptr;
    double *d_Kd = nullptr, *d_C = nullptr, *d_Chat = nullptr, *d_A = nullptr, *d_scal = nullptr, *d_in = nullptr;
    int* d_status = nullptr;
    size_t ring_elem = 4;
    long long host_step = 0, block_start = 0, noise_end = 0, last_fr_row = -1;
    bool noise_valid = false, have_kernels = false;
    std::vector<double> Kd, A;
    double a = 1.0, b = 1.0, spec_min = 0.0, clamped = 0.0;
    cudaGraphExec_t gexec = nullptr;
    bool graph_failed = false;
    int graph_mode = 0;  // 0 none, 1 gated rebuild kernels, 2 conditional rebuild node
    std::string msg;
    gld_status latched = GLD_OK;
    std::vector<int> int2ext;  // caller's index of the particle stored at k
    int* d_int2ext = nullptr;
    // recursive memory form: FP64 discrete weights w_a[m] of every
    // accumulator (kept from gld_set_kernels for the fit), mode tables, the
    // auxiliary sums, and whether they must be rebuilt from the ring
    std::vector<double> wts;
    float4* d_mcoef = nullptr;
    float2* d_mw = nullptr;
    float2* d_Y = nullptr;
    double* d_mz = nullptr;
    bool modes_dirty = false;
    // pair-correlated noise: filter taps [deg + 1][la], the blocks Z_1..Z_deg,
    // three Clenshaw vectors, and a word for the Gershgorin bound
    float* d_pntaps = nullptr;
    float* d_zblk = nullptr;
    float* d_bvec = nullptr;
    unsigned* d_rowsum = nullptr;
    // the Lanczos run that finds (and at each noise block checks) the
    // interval of the pair matrix's spectrum: four vectors [3][n_pad], two
    // sets of block partials, alpha/beta and the Ritz extremes; the interval
    double* d_lzpart = nullptr;
    float* d_lzv = nullptr;
    double* d_lzab = nullptr;
    double pn_lo = 0.0, pn_hi = 0.0;
    // pair-correlated noise by a Lanczos iteration per frequency: M
    // frequencies (Mp padded to 32), at most kmax iterations, the stopping
    // tolerance, device vectors and scalars, and the last step's statistics
    struct Krylov {
        int M = 0, Mp = 0, kmax = 0;
        double tol = 0.0;
        int window = 0, Mc = 0;  // the time window (one run per noise block), columns of the cosine part
        float *V = nullptr, *Y = nullptr, *cf = nullptr, *cosT = nullptr, *wgt = nullptr;
        double *part = nullptr, *alpha = nullptr, *beta = nullptr, *wc = nullptr;
        int* alive = nullptr;
        int last_iters = 0;
        double last_change = 0.0;
    } kry;
};

struct gld_batch {
    cudaStream_t st = nullptr, cap = nullptr;
    std::vector<gld_ctx*> members;
    char* d_plan = nullptr;  // descriptors, then tiles (stream-ordered allocation)
    size_t plan_cap = 0;
    char* h_stage[2] = {nullptr, nullptr};  // pinned staging of the plan upload
    size_t stage_cap[2] = {0, 0};
    cudaEvent_t stage_ev[2] = {nullptr, nullptr};
    int stage_k = 0;
    std::vector<std::pair<cudaGraphExec_t, cudaEvent_t>> retired;  // graphs possibly still running
    int tuning = 0;  // 0: re-time at every composition change; 1: when the column count moved 2x
    long long tuned_cols = 0;
    BatchPlan plan{};
    bool dirty = true;
    int schedule = -1;  // chosen convolution schedule (autotuned), -1: not yet
    double schedule_ms[4] = {0, 0, 0, 0};
    cudaGraphExec_t gexec = nullptr;
    std::vector<SysDesc> snap;  // member descriptors the plan was built from
    std::string msg;
};

namespace gld {
// Interprets the device error bits of a context as its synchronizing calls do
// (latching device failures); returns the latched status.
gld_status ctx_check_err(gld_ctx* c, unsigned err);
// Derived step parameters and cell count of a system (no device work).
void ctx_derive(const gld_params* p, StepParams& P, int& ncells);
// Device bytes a context holds after gld_create + gld_set_kernels with Q pair
// and Qs self-difference terms on nr table points (num_sms: of the device).
size_t ctx_bytes_needed(const gld_params* p, int Q, int Qs, int nr, int num_sms);
// Device bytes gld_set_pair_noise(degree K, Gershgorin bound) adds to them:
// the K + 1 filters, the blocks Z_1 .. Z_K, the Clenshaw vectors and the
// row-sum word.
size_t pn_bytes_needed(const gld_params* p, int K);
// [n][3] doubles in the caller's order from float4 rows in internal order.
void ctx_to_caller(const gld_ctx* c, const float4* h, double* dst);
}  // namespace gld
