// Internal declarations shared by the libsdmd translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sdmd.h"

namespace sdmd {

// Ring slots are padded to a multiple of this many bytes; the padding is zero
// and is never written, so kernels may process whole units.
constexpr int64_t kSlotAlign = 4096;

// Gram-row kernel geometry (gram_row.cu).
constexpr int kGrThreads = 256;
constexpr int kGrWarps = kGrThreads / 32;

// Device-side status word values (mirrors the public codes).
constexpr int kDevOk = 0;
constexpr int kDevRank = 1;      // an eigensolver reached its iteration cap
constexpr int kDevTimeout = 2;   // a bounded wait gave up
constexpr int kDevRange = 4;     // a sparse coefficient index was outside [0, n)

struct GramRowArgs {
  const uint8_t* ring;   // slot j starts at ring + j * slot_bytes
  int64_t slot_bytes;    // multiple of kSlotAlign
  int64_t chunk;         // bytes per chunk, multiple of 4096
  int32_t nblk;          // chunks; nblk * chunk >= slot_bytes
  int32_t c;             // resident snapshots (after this push)
  int32_t s_first;       // physical slot of the oldest resident snapshot;
                         // the window is slots s_first, s_first+1, ... (mod m)
  int32_t s_new;         // slot holding the new snapshot
  int32_t m;             // G is m x m
  void* partials;        // [m][nblk] per-chunk partial sums (FP64 or int64)
  unsigned int* ticket;  // two words, zero between launches: CTAs finished, chunks taken
  void* G;               // m x m, double (f32) or int64 (u8), physical slots
  int* status;           // device status word (kDevTimeout on an expired wait)
};

// Gram rows/columns of the k newest uint8 snapshots against the window
// (k = c: the full Gram) on the tensor cores, exact. The host call splits
// the targets into groups of at most 64 and pairs each group with blocks of
// older snapshots; one kernel launch covers one (group, block) pair.
struct GramFullArgs {
  const uint8_t* ring;
  int64_t slot_bytes;
  int64_t n;
  int32_t m;             // ring modulus (G is m x m, physical slots)
  int32_t start;         // physical slot of the oldest resident snapshot
  int32_t c;             // resident snapshots
  int32_t k;             // targets: the k newest (k = c: the whole Gram)
  long long* partials;   // [kGramFullMaxCtas][128][128] per-CTA sums
  unsigned* sched;       // chunk counter, zero between launches
  long long* G;
  int* status;
  // one launch (set by launch_gram_full_tc): tile rows = targets (window time
  // indices t_tgt .. t_tgt + k - 1), the ones row, then nold older snapshots
  // (t_old .. t_old + nold - 1); k + 1 + nold <= 128
  int32_t t_tgt = 0, t_old = 0, nold = 0;
};
constexpr int kGramFullMaxCtas = 160;
constexpr int kGramFullMaxTargets = 64;
// Launches the kernels of every (target group, older block) pair on `st`;
// cudaErrorNotSupported outside 1 <= k <= c <= SDMD_MAX_M.
cudaError_t launch_gram_full_tc(const GramFullArgs& a, int* ctas_out, cudaStream_t st);

// Gram rows/columns of FP32 snapshots on the tensor cores in BF16x3 split
// precision: one launch pairs k <= 64 target snapshots (window time indices
// t_tgt ..) with themselves and with nold older ones (t_old ..), k + nold <= 128.
struct GramF32Args {
  const uint8_t* ring;
  int64_t slot_bytes;
  int64_t n;
  int32_t m;             // ring modulus (G is m x m doubles, physical slots)
  int32_t start;         // physical slot of window time index 0 (the oldest)
  int32_t t_tgt, k;      // target rows
  int32_t t_old, nold;   // older rows
  int32_t split;         // 3: three bf16 terms, six products; 2: two terms, three products
  float2* partials;      // [kGramF32MaxCtas][128][64] per-CTA (hi, lo) sums
  double* G;
  int* status;
};
constexpr int kGramF32MaxCtas = 160;
constexpr int kGramF32MaxTargets = 64;
// All launches for the k newest of c resident snapshots (k = c: the whole
// Gram) on `st`; `launches` receives the number of main-kernel launches.
cudaError_t launch_gram_f32_tc(const GramF32Args& base, int c, int k, int num_sms, int* launches, cudaStream_t st);
int gram_f32_tc_ctas(int64_t n, int num_sms);

// The k newest of c resident FP32 snapshots (k <= 16, c <= 256) against the
// whole window on the CUDA cores: FP32 products, 64-position FP32 runs,
// compensated sums, FP64 over CTAs (gram_f32_simt.cu).
struct GramF32SimtArgs {
  const uint8_t* ring;
  int64_t slot_bytes;
  int64_t n;
  int32_t m;             // ring modulus (G is m x m doubles, physical slots)
  int32_t start;         // physical slot of window time index 0 (the oldest)
  int32_t c, k;          // rows: time indices 0..c-1; targets: the last k
  float2* partials;      // [kGramF32MaxCtas][256][16] per-CTA (hi, lo) sums
  double* G;
};
constexpr int kGramF32SimtMaxTargets = 16;
cudaError_t launch_gram_f32_simt(const GramF32SimtArgs& a, int num_sms, cudaStream_t st);

// One snapshot's Gram row inside a batched launch (fields as in GramRowArgs).
struct RowJob {
  const uint8_t* ring;
  int64_t slot_bytes;
  int64_t chunk;
  void* partials;
  unsigned int* ticket;  // chunks finished (word 0), zero between launches
  void* G;
  int32_t nblk, c, s_first, s_new, m;
  int32_t mode;          // 0 uint8, 1 float32, 2 complex64, 3 float32 with FP64 products
  int32_t item0;         // first work item of this job in the batch
};
constexpr int kMaxBatchJobs = 64;
struct BatchArgs {
  RowJob job[kMaxBatchJobs];
  int32_t njobs;
  int32_t nitems;        // sum of the jobs' chunk counts
  unsigned int* grab;    // two words, zero between launches: items taken, CTAs finished
  int* status;           // status word of the first handle
};
cudaError_t launch_gram_rows_batched(const BatchArgs& a, cudaStream_t st);
// Launch configuration of the batched kernel for a graph kernel node (func,
// grid, block, shared memory; kernelParams left to the caller); sets the
// kernel's shared-memory attribute on first use.
cudaError_t batched_kernel_config(const BatchArgs& a, cudaKernelNodeParams* p);

// One batched push, planned: the handles' deferred work flushed, ring readers
// waited for, the ingest copies and the batch arguments filled in; no
// handle's ring moves yet. The caller issues the copies, then the batched
// kernel (directly or as graph nodes), on `st`, and then calls
// push_many_finish with how many of the leading copies were enqueued and
// whether the kernel was: every handle whose snapshot reached its ring
// advances (with its own Gram-row pass if the batched kernel did not run),
// the others stay as they were.
struct BatchPlan {
  BatchArgs args;
  int ncopies;
  void* dst[kMaxBatchJobs];
  const void* src[kMaxBatchJobs];
  size_t bytes[kMaxBatchJobs];
};
int push_many_plan(sdmd_t const* hs, const void* const* xs, int count, cudaStream_t st, BatchPlan* plan);
int push_many_finish(sdmd_t const* hs, int count, int copied, bool launched, cudaStream_t st);

// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device. The attribute belongs to a device, so the level reached is
// kept per (kernel, device); thread-safe.
cudaError_t smem_optin(const void* func, size_t bytes);

// Device bytes of a depth-1 dense handle (admission by footprint).
int64_t handle_device_bytes(int64_t n, int32_t m, int32_t dtype, int num_sms);

// Gram row for one pushed snapshot; launches one kernel on `st`.
// f64_ref: FP32 snapshots with FP64 products and sums (SDMD_OPT_F32_FP64).
cudaError_t launch_gram_row(int dtype, bool f64_ref, const GramRowArgs& a, cudaStream_t st);

// Schedule of the Gram-row kernel: a function of slot size and SM count only,
// so that every entry of G sees the same summation order.
void gram_row_schedule(int64_t slot_bytes, int num_sms, int64_t* chunk, int32_t* nblk);
// The same with a given number of chunks per SM (the autotuner's candidates).
void gram_row_schedule_k(int64_t slot_bytes, int num_sms, int chunks_per_sm, int64_t* chunk, int32_t* nblk);

struct ModesArgs {
  const void* G;        // m x m physical (double or int64)
  int32_t g_is_int;     // 1: int64 entries
  int32_t m;            // stride of G and modulus of its slot indices
  int32_t ws_m;         // window length the workspace `ws` was laid out for
  int32_t c;            // resident snapshots (>= 3)
  int32_t start;        // physical slot of the oldest resident snapshot (0 <= start < m)
  int32_t r_req;        // requested modes (1 <= r_req <= c-1)
  double* ws;           // workspace (modes_ws_doubles(m) doubles)
  int* status;          // device status word (sticky error bits)
  int* r_dev;           // kept rank (device int)
  // Complex windows through the real df64 eigensolver: with embed_cx = 1 the
  // real modes kernel reads G as complex128, runs its phases 0-4 on the real
  // symmetric embedding [[Re G_X, -Im G_X], [Im G_X, Re G_X]] (2p x 2p, every
  // eigenvalue of G_X twice) for r_req = 2K eigenpairs, and hands the K
  // complex eigenpairs (lambda, x = u + i v from each pair's first vector
  // [u; v]) to the complex kernel's workspace; cx_pre = 1 makes the complex
  // kernel take them instead of running its Jacobi sweeps.
  int32_t embed_cx = 0;
  int32_t cx_pre = 0;
};

// Doubles of workspace needed by the modes kernel for window length m.
int64_t modes_ws_doubles(int m);

// Offsets (in doubles) of the named arrays inside the modes workspace.
struct ModesLayout {
  int64_t A, GXY, HV, d, e, lam, Z, V, Y, At, Hc, Qc, Wc, M, Mf, sig, lamout, tmp, lu, clk;
  int64_t bamp;   // r complex128 mode amplitudes b (Sec. 3.3), then the background index (as double)
  int64_t urec;   // p x 2 floats: reconstruction weights (hi, lo) of X' columns
  int64_t Mu;     // p x r floats: V Sigma^-1 for the POD modes
  int64_t cx;     // complex windows: six p x p complex128 arrays (V of sdmd_svd at the sixth)
  int64_t total;
};
__host__ __device__ ModesLayout modes_layout(int m);

cudaError_t launch_modes_small(const ModesArgs& a, cudaStream_t st);
// The real-window eigensolvers of several handles in one launch (one CTA per
// job; each job exactly as launch_modes_small would run it alone).
constexpr int kMaxModesJobs = 64;
struct ModesBatch {
  ModesArgs job[kMaxModesJobs];
  int32_t count;
};
cudaError_t launch_modes_batch(const ModesBatch& b, cudaStream_t st);
// The same outputs for complex windows (G complex128 Hermitian): FP64 Jacobi
// for G_X, complex A~, W, M and amplitudes.
cudaError_t launch_modes_complex(const ModesArgs& a, cudaStream_t st);
// Whether a complex window of c snapshots and rank r can take the embedded
// df64 path (its working set fits what that path may use).
bool modes_embed_ok(int c, int r);

struct PhiArgs {
  const uint8_t* ring;
  int64_t slot_bytes;
  int64_t n;
  int32_t dtype;
  int32_t m;
  int32_t start;        // physical slot of the oldest resident snapshot (0 <= start < m)
  int32_t p;            // c-1 columns of X'
  int32_t r;            // requested modes (output columns)
  const float* Mf;      // p x 2r  (re, im) of V Sigma^-1 W, FP32
  const int* r_dev;     // kept rank; columns >= *r_dev are written as zero
  float* phi;           // n x r complex64, column-major
  int* status;          // device status word
  int32_t tensor;       // 1: use the tensor-core kernel where it applies
  unsigned* sched;      // kPhiSchedWords zeroed words: per-pass tile counters, CTA-done counter
  int32_t xoff = 1;     // first window column read: 1 = X' (Phi), 0 = X (POD modes)
  int32_t real_out = 0; // 1: Mf is p x r real, phi is n x r FP32 (CUDA-core kernel)
  // Fused Gram row (tensor-core uint8 kernel): the staged rows continue past
  // X' to ktot slots in time order (slots start + 1 .. start + ktot), the
  // last being the new snapshot; rows g0 .. ktot - 1 are the new window, and
  // each CTA adds its exact sums of <x_u, x_new> to gpart[cta][u - g0].
  int32_t fuse = 0;
  int32_t ktot = 0, g0 = 0;
  long long* gpart = nullptr;
  // 1: modes per tensor-core pass fitted to r (10 when r <= 10: N = 64),
  // 0: always 16 modes per pass (N = 96); both give the same values
  int32_t fit_modes = 1;
};
// Per-CTA partial capacity of the fused Gram row (CTAs x window slots).
constexpr int kFusedMaxCtas = 160;
constexpr int kFusedReserveSms = 4;   // SMs the fused pass leaves to concurrent eigensolvers
constexpr int kPhiSchedPasses = 16;                 // mode passes of 16 (r <= 256)
constexpr int kPhiSchedWords = kPhiSchedPasses + 1;

cudaError_t launch_phi(const PhiArgs& a, cudaStream_t st);
// Phi of one frame and the Gram row of a later snapshot in one pass over the
// union of their windows (uint8, tensor cores), then G's new row and column
// (int64, physical slots: s_new, and slot0 + jj for window index jj).
cudaError_t launch_phi_fused(const PhiArgs& a, long long* G, int32_t gm, int32_t s_new, int32_t slot0,
                             cudaStream_t st);
// Mu[j][k] = V[k][j] / sigma_k (zero beyond the kept rank), then
// U = X Mu with the real CUDA-core Phi kernel (xoff = 0, real_out = 1).
cudaError_t launch_pod_modes(const PhiArgs& a, const double* V, const double* sig, float* Mu, cudaStream_t st);

struct ReconArgs {
  const uint8_t* ring;
  int64_t slot_bytes;
  int64_t n;
  int32_t dtype;        // SDMD_U8 or SDMD_F32
  int32_t m;            // ring modulus
  int32_t start;        // physical slot of the oldest snapshot of the modes window
  int32_t p;            // columns of X'
  int32_t R;            // modes requested in the modes call (stride of Mf)
  const float* Mf;      // p x 2R (re, im) of M = V Sigma^-1 W
  const double* lamout; // R complex eigenvalues
  const double* bamp;   // R complex amplitudes
  const double* bgi;    // background mode index (stored as double)
  const int* r_dev;     // kept rank
  int64_t t;            // time index, 0 = x_1
  int32_t what;         // SDMD_RECON_*
  float* urec;          // workspace: p x 2 floats
  float* out;           // n floats, 16-byte aligned
  int32_t xt_slot;      // physical slot of x_t (foreground), -1 otherwise
  double slow_tol;      // SDMD_RECON_*_SLOW: modes with |log lambda| <= slow_tol
};
cudaError_t launch_reconstruct(const ReconArgs& a, cudaStream_t st);
// tcgen05 kernel for uint8 windows; cudaErrorNotSupported outside its shapes
cudaError_t launch_phi_tc(const PhiArgs& a, cudaStream_t st);

struct SparseRowArgs {
  const int* idx_ring;       // slot j's indices at idx_ring + j * nnz_max
  const float2* val_ring;    // slot j's complex64 values
  int nnz_max;
  const int* tag;            // lookup table tags (length n)
  const float2* tval;        // lookup table values (length n)
  int64_t n;
  int stamp;                 // tag value of the new snapshot's entries
  int c, s_first, s_new, m;
  int nnz[SDMD_MAX_M];          // entries per physical slot
  int chunk_start[SDMD_MAX_M];  // first CTA of window slot jj
  int nblk;
  double2* partials;         // one per CTA
  unsigned int* ticket;
  void* G;                   // m x m complex128
};

// CTAs a snapshot with nnz entries takes in the sparse row kernel.
int sparse_chunks(int nnz);
cudaError_t launch_sparse_scatter(const int* idx, const float2* val, int nnz, int64_t n, int stamp, int* tag,
                                  float2* tval, int* status, cudaStream_t st);
cudaError_t launch_sparse_row(const SparseRowArgs& a, cudaStream_t st);

// Modes of a Fourier-sparse window in coefficient space (compressed Phi-hat).
struct FourierPhiArgs {
  const int* idx_ring;       // slot j's sorted indices at idx_ring + j * nnz_max
  const float2* val_ring;    // slot j's complex64 values
  int nnz_max;
  int nnz[SDMD_MAX_M];       // entries per physical slot
  int m;                     // ring modulus
  int start;                 // physical slot of the oldest resident snapshot
  int p;                     // X' columns: slots start + 1 .. start + p
  int r, R;                  // modes to write; stride of Mf (modes of the modes call)
  const float* Mf;           // p x 2R (re, im) of M = V Sigma^-1 W
  int64_t n;                 // coefficients per snapshot
  unsigned* bitmap;          // ceil(n / 32) words
  unsigned long long* prefix;// ceil(n / 32) exclusive popcount prefix
  unsigned long long* count; // union size
  int* idx_out;              // cap sorted coefficient indices
  float2* phi_out;           // cap x r complex64, column-major (leading dimension cap)
  int64_t cap;
};
// Marks and counts the union support; with `rows`, also writes idx_out and
// phi_out (the first min(count, cap) entries).
cudaError_t launch_fourier_phi(const FourierPhiArgs& a, bool rows, cudaStream_t st);

// Records `msg` as this thread's sdmd_last_error() text; returns `code`.
int set_last_error(int code, const char* msg);

}  // namespace sdmd
