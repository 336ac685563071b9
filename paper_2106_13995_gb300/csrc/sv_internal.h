// Internal declarations shared by the library's translation units.
// Host-side structures (state handle, programs) and the device-side program
// format read by the tile-pass kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <complex>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/sv_api.h"

namespace sv {

using cd = std::complex<double>;

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------
sv_status set_error(sv_status st, const std::string &msg);
sv_status cuda_error(cudaError_t e, const char *what);
extern std::atomic<uint64_t> g_launches;

#define SV_CUDA(call)                                            \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return ::sv::cuda_error(e_, #call);   \
  } while (0)

#define SV_TRY(call)                      \
  do {                                    \
    sv_status s_ = (call);                \
    if (s_ != SV_OK) return s_;           \
  } while (0)

// ---------------------------------------------------------------------------
// device program format for tile passes
// ---------------------------------------------------------------------------
enum TileOpKind : uint8_t {
  TOP_DENSE = 0,     // v <- U v on local targets (k = 1..6), local + global controls
  TOP_DIAG = 1,      // v[l] <- d[r(l)] v[l], r over local targets
  TOP_GRAD = 2,      // acc[slot] += Im <v1 | G v0>, G = X/Y/Z/P1(-2) on one local target
  TOP_PAULI = 3,     // v1[l ^ xm] += c * phase * (-1)^{popcount(l & zm)} v0[l]
  TOP_ZERO = 4,      // v1 <- 0
  TOP_DOT = 5,       // acc[slot] += Re <v0 | v1>
  TOP_TC = 6,        // 5-qubit dense block on the tensor cores (12-qubit tiles)
  TOP_PERM = 7,      // permutation block (k = 1..3): member y moves to member perm[y]; controls as TOP_DENSE
  TOP_GRADU = 8      // TOP_GRAD then the 1-qubit matrix (per-batch pool) on both vectors, in one sweep
};

// 32-byte op descriptor; matrices live in a separate pool.
struct TileOp {
  uint8_t kind;
  uint8_t k;          // number of targets
  uint8_t vmask;      // bit0: apply to v0, bit1: apply to v1
  uint8_t gen;        // TOP_GRAD generator: 1=X 2=Y 3=Z 4=diag(0,-2)
  uint8_t t[6];       // local target positions, matrix bit order
  uint8_t tbpos[6];   // dense/diag: local position of thread-index bit i (4 bits each, i < 9)
  uint32_t lcmask;    // local control mask (bits of the tile-local index)
  uint32_t mat;       // offset (complex entries) into the matrix pool; TOP_PAULI: coeff index
  uint32_t gcmask_lo; // controls outside the tile, as a mask of global bits (low 32)
  uint16_t gcmask_hi; // ... bits 32..47
  int16_t slot;       // accumulator slot (TOP_GRAD / TOP_DOT); TOP_PAULI: x mask (local)
};
static_assert(sizeof(TileOp) == 32, "TileOp must stay 32 bytes");

// Per-pass launch description (passed by value as a kernel parameter).
constexpr int kMaxQ = 34;
constexpr uint8_t kGenBatchMat = 0x80;   // TileOp.gen flag: matrix from the per-batch pool
constexpr uint8_t kGenInline = 0x40;     // TileOp.gen flag: matrix in the launch's parameter block

// Parameter block of a complex64 single-vector tile pass: its op list and
// the matrices of its 1-3 qubit dense blocks, read by every CTA with
// warp-uniform loads (matrices as row pairs, see dense_pairs).  Passes that
// do not fit keep the global copies.
constexpr int kInlOps = 48;
constexpr int kInlMat = 3200;    // complex64 entries
// groups per trip of the packed complex64 blocks from the parameter block
constexpr int pairs_groups(int k) { return k <= 2 ? 4 : 2; }
// Per-op set-up of a parameter-block dense block, computed on the host for
// the launch's thread count: the swizzled member offsets, the swizzled trip
// offsets of the first trips and of a trip's groups, and the trip map.
struct OpPre {
  uint32_t soff[8];    // swb of the member offsets (the K target bits)
  uint32_t dh[4];      // swb(l(h T)), h < groups per trip
  uint32_t tc[4];      // swb(l(c0 T)) for the first four trips c0 = 0, G, 2G, 3G
  uint32_t tm_hi;      // TripMap
  uint32_t tm_shift;
};
// OpPre of a 1-3 qubit dense op for a launch with `threads` threads (k_tile.cu)
void fill_op_pre(const TileOp &op, int threads, OpPre &pre);
struct TileInline {
  uint32_t nops, nmat;
  TileOp ops[kInlOps];
  OpPre pre[kInlOps];
  float2 mats[kInlMat];
};
// TilePass.flags: this entry is not a tile pass but one dense block of L = 5
// or 6 qubits on the tensor cores; hi_pos[0..L) hold its targets, mat0 the
// 16-byte index of its packed operand in the matrix pool, bits 9..10 the
// sv_prec mode (6-qubit blocks: split-BF16 only).
constexpr uint32_t kPassTC = 0x100;
// TilePass.flags: the pass contains TOP_TC ops (allocate TMEM); mode in bits 9..10
constexpr uint32_t kPassHasTC = 0x8;
// TilePass.flags: a permutation pass with no ops: every amplitude of a tile
// moves by a gather table (16-byte index mat0 of its block in the matrix
// pool; k_tile_tperm)
constexpr uint32_t kPassTable = 0x800;
constexpr int kTcTileM = 12;          // tile size that gives M = 128 groups for a 5-qubit block
size_t tc_tile_smem(sv_prec mode);    // shared memory of a 12-qubit tile pass with TOP_TC ops
struct TilePass {
  int32_t n;              // state qubits
  int32_t m;              // tile qubits
  int32_t L;              // low qubits included in every tile (contiguous segment 2^L)
  int32_t nops;
  int8_t hi_pos[kMaxQ];   // global position of local bit L + j
  int8_t out_pos[kMaxQ];  // sorted global positions not in the tile (n - m of them)
  uint32_t flags;         // bit0: v1 is zeroed by the pass, do not load it
  uint32_t nvec;          // 1 or 2 vectors per tile
  uint32_t mat0;          // tensor-core entries (kPassTC): 16-byte index of the operand in the pool
  uint32_t pad0;
  const TileOp *ops;      // device: this pass's ops
  const void *mats;       // device: shared matrix pool
  const void *pmats;      // device: per-batch matrix pool
  uint64_t pmats_stride;  // complex entries per batch item
  const double *coeffs;   // device: TOP_PAULI coefficients
  double *acc;            // device: FP64 accumulators
  uint64_t acc_stride;    // doubles per batch item
  void *const *tbl0;      // device: per-batch pointers of vector 0 (or null)
  void *const *tbl1;      // device: per-batch pointers of vector 1 (or null)
  void *v0;               // vector 0 when tbl0 is null
  void *v1;               // vector 1 when tbl1 is null
  uint32_t *err;          // error flag for bounded waits (TOP_TC)
};

// Arguments of the persistent batch kernel (all pointers are device memory).
struct PersistArgs {
  const TilePass *passes;            // ndesc pass descriptors, wave-major order
  const unsigned long long *first_item;  // first queue item (chunk) of each descriptor
  const int32_t *dep;                // descriptor this one waits for, or -1
  const uint32_t *ntiles;            // tiles of each descriptor
  const uint32_t *chunk;             // tiles per queue item of each descriptor
  uint32_t *done;                    // finished tiles per descriptor (zeroed before launch)
  unsigned long long *next_item;     // queue head (zeroed before launch)
  uint32_t *err;                     // set to 1 when a bounded wait runs out
  unsigned long long total_items;    // queue items (chunks)
  uint32_t ndesc;
  uint32_t pad;
  uint64_t spin_limit;               // polls per wait
};

// ---------------------------------------------------------------------------
// host-side gate representation and planners
// ---------------------------------------------------------------------------
struct Gate {
  std::vector<int> targets;    // matrix bit j <-> targets[j]
  std::vector<int> controls;
  std::vector<cd> U;           // 2^k x 2^k row-major
  int param_gate = -1;         // sv_gate for parametric gates (adjoint generator)
  int param = -1;              // parameter index or -1
  bool fixed_structure = false;  // never fuse (parametric in batched programs)
  int inst = -1;               // parametric instance index (per-batch matrix table)
  int grad_gen = 0;            // >0: gradient probe Im<v1|G v0> instead of a gate
  int grad_slot = -1;
};

struct Block {
  std::vector<int> qubits;     // targets (matrix bit order)
  std::vector<int> controls;   // remaining controls (unfused controlled gates)
  std::vector<cd> U;
  bool diag = false;
  bool fusable = true;
  int param = -1;              // parametric single gate (batched / gradient)
  int param_gate = -1;
  int kind = TOP_DENSE;        // TOP_DENSE / TOP_GRAD / ...
  int gen = 0;
  int vmask = 1;
  int slot = -1;
  int inst = -1;               // parametric instance (per-batch matrix)
  double coeff = 0;
  uint64_t xmask = 0, zmask = 0;
};

// gates.cpp
int gate_arity(int gate);                                    // -1 unknown
bool gate_matrix(int gate, const double *angles, std::vector<cd> &U);
int gate_generator(int gate);                                // 1=X 2=Y 3=Z 4=diag(0,-2), 0 none
sv_status circuit_to_gates(const sv_circuit *c, const double *params, int n,
                           std::vector<Gate> &out, bool keep_params_unfused);
std::vector<cd> adjoint_of(const std::vector<cd> &U, int k);
// caller matrices checked for unitarity (SV_DEBUG builds, or SV_CHECK_UNITARY=1)
constexpr double kUnitaryTol = 1e-10;
bool unitarity_checks();
double unitarity_error(const std::vector<cd> &U, int k);

// planner.cpp
std::vector<Block> fuse(const std::vector<Gate> &gates, int fusion_k);
struct PassPlan {
  std::vector<int> S;          // tile qubits: S[0..L) = 0..L-1, then sorted high qubits
  std::vector<Block> ops;
};
int max_targets(const std::vector<Block> &blocks);
// Shrink L (keeping >= lmin) or grow m (up to mmax, at most n) so that every
// block's targets fit one tile.  False if impossible.
bool fit_tile(const std::vector<Block> &blocks, int n, int lmin, int mmax, int &m, int &L);
// Empty result when some block cannot fit a tile of m qubits with L fixed low
// qubits (callers size m and L with fit_tile first).
std::vector<PassPlan> plan_passes(const std::vector<Block> &blocks, int n, int m, int L,
                                  int max_ops, int max_mat_entries);
// Blocks of the planned passes in execution order, with blocks of a pass
// merged where commuting lets them meet and the union has at most K qubits.
std::vector<Block> merge_in_passes(const std::vector<PassPlan> &passes, int K);

// ---------------------------------------------------------------------------
// state handle
// ---------------------------------------------------------------------------
struct DeviceProgram {
  std::vector<TilePass> passes;
  std::vector<TileOp> ops;
  std::vector<uint8_t> mats;      // matrix pool bytes (dtype of the state)
  std::vector<double> coeffs;     // TOP_PAULI coefficients
  uint32_t n_slots = 0;
};

}  // namespace sv

// streams over which a batched call spreads its wide states
constexpr int kFanStreams = 4;

struct sv_state {
  int n = 0;
  sv_dtype dt = SV_C64;
  void *amps = nullptr;
  size_t amps_bytes = 0;
  char *ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int sm_count = 0;
  // pinned host staging
  char *pinned = nullptr;
  size_t pinned_bytes = 0;
  cudaEvent_t staged = nullptr;     // last upload from `pinned` finished
  cudaStream_t capture = nullptr;   // library-owned stream used only to record CUDA graphs
  // library-owned streams and fork/join events over which a batch spreads
  // its independent wide states (sv_apply_circuit_batch), made on first use
  cudaStream_t fan[kFanStreams] = {};
  cudaEvent_t fan_fork = nullptr;
  cudaEvent_t fan_join[kFanStreams] = {};
  uint64_t resident = 0;            // serial of the program in the workspace program area (0: none)
  // the state is known to be basis_amp |basis_index>: set by sv_set_basis,
  // kept by circuits of permutation and phase gates, cleared by every other
  // write to the amplitudes (and by sv_mark_modified)
  bool basis_known = false;
  uint64_t basis_index = 0;
  std::complex<double> basis_amp = 1.0;
};

namespace sv {

// workspace layout (byte offsets)
constexpr size_t kWsCtrl = 0;                    // flags, counters, scalars
constexpr size_t kWsCtrlBytes = 256 << 10;
constexpr size_t kWsProg = kWsCtrlBytes;         // uploaded programs
constexpr size_t kWsProgBytes = 8 << 20;
constexpr size_t kWsRed = kWsProg + kWsProgBytes;  // reduction / sampling area
size_t red_bytes(int n);
constexpr size_t kPinnedBytes = kWsProgBytes + kWsCtrlBytes;

size_t amp_bytes(sv_dtype dt);
int lmin(sv_dtype dt);            // low qubits a tile must keep contiguous (16-byte copies)
int mmax(sv_dtype dt, int nvec);  // largest tile that fits shared memory
constexpr size_t kWsScalars = 0;            // FP64 result slots (4 KB)
constexpr size_t kWsErrFlag = 3072;         // uint32 device error bits (below)
constexpr uint32_t kErrWaitTimeout = 1u;     // a bounded device wait ran out
constexpr uint32_t kErrNoInlineBlock = 2u;   // a parameter-block tile pass met a block outside it
constexpr size_t kWsGateMat = 64 << 10;     // single-gate matrix scratch (k >= 4)

// program building / upload / launch (sv_api.cu)
struct BuildCtx {
  sv_dtype dt;
  int n, m, L;
  uint32_t nvec;
  uint32_t flags;
  int prec = SV_PREC_PLAIN;   // mode of TOP_TC ops
};
sv_status emit_pass(DeviceProgram &prog, const PassPlan &P, const BuildCtx &b,
                    std::vector<uint32_t> &op0s, const std::vector<int> &batch_mat_off);
struct ProgLayout {
  size_t ops_off, mats_off, coeffs_off, tbl_off, pmats_off, end;
};
ProgLayout layout_of(const DeviceProgram &p, size_t tbl_bytes, size_t pmats_bytes);
sv_status stage_upload(sv_state *s, const std::vector<std::pair<const void *, size_t>> &parts,
                       const std::vector<size_t> &offs, size_t total);
sv_status stage_upload_to(sv_state *s, void *dst, const std::vector<std::pair<const void *, size_t>> &parts,
                          const std::vector<size_t> &offs, size_t total);
struct LaunchEnv {
  int batch = 1;
  void *const *tbl0 = nullptr;
  void *const *tbl1 = nullptr;
  void *v0 = nullptr, *v1 = nullptr;
  const void *pmats = nullptr;
  uint64_t pmats_stride = 0;
  double *acc = nullptr;
  uint64_t acc_stride = 0;
};
sv_status launch_program(sv_state *s, const DeviceProgram &p, const ProgLayout &L,
                         const std::vector<uint32_t> &op0s, const LaunchEnv &E, cudaStream_t st = nullptr);
struct Opts {   // all int: hashed as key bytes, so no padding
  int fusion_k, tile_m, L, prec, mode;
  int tc_in_tile = 0;
};
Opts resolve(const sv_state *s, const sv_options *o, int nvec);
// Fill fusion_k / tile_m that the caller left at 0 from the autotuner's
// cache for this circuit's shape (sv_batch.cu).
void tuned_options(const sv_state *s, const sv_circuit *c, const sv_options *opt, Opts &o);
// ---------------------------------------------------------------------------
// program caches
// ---------------------------------------------------------------------------
// Key material of a cached program: every byte that determines it (circuit
// ops and matrices, parameters, resolved options, dtype).  Lookups hash it
// and compare it byte for byte on a hash hit, so a collision never returns
// another circuit's program.
struct KeyBytes {
  std::vector<uint8_t> b;
  void bytes(const void *p, size_t n) {
    const uint8_t *q = static_cast<const uint8_t *>(p);
    b.insert(b.end(), q, q + n);
  }
  template <typename T> void val(const T &v) { bytes(&v, sizeof(T)); }
  uint64_t hash() const;
};
// key material of a circuit (ops, the matrices its MATRIX ops use)
void circuit_key(KeyBytes &k, const sv_circuit *c);
uint64_t next_program_serial();

// A bounded, thread-safe cache of immutable programs per state handle.
// Entries are shared: a caller holding one keeps it alive even after the
// cache evicts it (oldest first once more than `limit` are held).
template <class V> class ProgCache {
 public:
  explicit ProgCache(size_t limit) : limit_(limit) {}
  std::shared_ptr<const V> find(const void *owner, const KeyBytes &k, uint64_t h) {
    std::lock_guard<std::mutex> lk(mu_);
    auto r = map_.equal_range(h);
    for (auto it = r.first; it != r.second; ++it)
      if (it->second.owner == owner && it->second.key == k.b) return it->second.val;
    return nullptr;
  }
  // Insert v unless an equal key is present; returns the cached entry.
  std::shared_ptr<const V> insert(const void *owner, const KeyBytes &k, uint64_t h, std::shared_ptr<const V> v) {
    std::lock_guard<std::mutex> lk(mu_);
    auto r = map_.equal_range(h);
    for (auto it = r.first; it != r.second; ++it)
      if (it->second.owner == owner && it->second.key == k.b) return it->second.val;
    const uint64_t seq = ++seq_;
    map_.emplace(h, Entry{owner, k.b, v, seq});
    order_.emplace_back(h, seq);
    while (map_.size() > limit_ && !order_.empty()) {
      erase_locked(order_.front().first, order_.front().second);
      order_.pop_front();
    }
    return v;
  }
  void drop_owner(const void *owner) {
    std::lock_guard<std::mutex> lk(mu_);
    for (auto it = map_.begin(); it != map_.end();) it = it->second.owner == owner ? map_.erase(it) : std::next(it);
  }
  size_t set_limit(size_t n) {
    std::lock_guard<std::mutex> lk(mu_);
    const size_t old = limit_;
    if (n > 0) limit_ = n;
    return old;
  }
  size_t size() {
    std::lock_guard<std::mutex> lk(mu_);
    return map_.size();
  }

 private:
  struct Entry {
    const void *owner;
    std::vector<uint8_t> key;
    std::shared_ptr<const V> val;
    uint64_t seq;
  };
  void erase_locked(uint64_t h, uint64_t seq) {
    auto r = map_.equal_range(h);
    for (auto it = r.first; it != r.second; ++it)
      if (it->second.seq == seq) {
        map_.erase(it);
        return;
      }
  }
  std::mutex mu_;
  std::unordered_multimap<uint64_t, Entry> map_;
  std::deque<std::pair<uint64_t, uint64_t>> order_;
  uint64_t seq_ = 0;
  size_t limit_;
};

// Cached plain-circuit program (one vector) and its lookup.
struct CachedProgram {
  DeviceProgram prog;
  std::vector<uint32_t> op0s;
  ProgLayout lay;
  std::vector<Block> blocks;   // for per-gate mode
  uint64_t serial = 0;         // unique per built program (workspace residency tag)
};
using ProgramRef = std::shared_ptr<const CachedProgram>;
constexpr size_t kProgramCacheDefault = 2048;
sv_status get_program(sv_state *s, const sv_circuit *c, const double *params, const sv_options *opt,
                      ProgramRef *out, Opts *o_out);
sv_status upload_program(sv_state *s, const CachedProgram &cp);
// Set a kernel attribute once per (kernel, device, attribute, value); thread-safe.
sv_status func_attr_once(const void *fn, int device, cudaFuncAttribute attr, int value);
void drop_graphs(const sv_state *s);
void drop_adjoint_programs(const sv_state *s);

// kernels (launchers), all enqueue on s->stream
sv_status launch_set_basis(sv_state *s, uint64_t index);
// psi[from] := 0, psi[to] := a (one thread; the state is a basis state)
sv_status launch_move_basis(sv_state *s, uint64_t from, uint64_t to, cd a);
// copy `bytes` (a multiple of 16, both pointers 16-byte aligned and
// addressable by the device: device memory or mapped page-locked host
// memory) by a grid-stride kernel on the state's stream
sv_status launch_copy16(sv_state *s, const void *src, void *dst, size_t bytes);
// Follow a basis state through gates that map it to a basis state times a
// phase (permutations, diagonal and monomial gates, with controls); false,
// leaving index and amp unspecified, as soon as one gate does not.
bool propagate_basis(const std::vector<Gate> &gates, uint64_t &index, cd &amp);
sv_status launch_scale(sv_state *s, double factor);
sv_status launch_dense_gate(sv_state *s, const std::vector<int> &targets,
                            const std::vector<int> &controls, const std::vector<cd> &U);
sv_status launch_diag_gate(sv_state *s, const std::vector<int> &targets,
                           const std::vector<int> &controls, const std::vector<cd> &d);
sv_status launch_norm(sv_state *s, double *out_dev_scalar);
sv_status launch_expect_group(sv_state *s, uint64_t xmask, const uint64_t *zm, const double *cf,
                              const int *ipow, int nt, double *out_dev);
sv_status launch_z_all(sv_state *s, double *out_dev);
sv_status zall_noalloc(const void *amps, int n, sv_dtype dt, double *out, cudaStream_t stream);
sv_status launch_sample_prepare(sv_state *s);
sv_status launch_sample_shots(sv_state *s, int64_t shot0, int64_t count, uint64_t seed, uint64_t *out_dev);
size_t sample_shot_offset(int n);
size_t scan_scratch_bytes(int n);   // prefix-scan scratch after the shot buffer
int64_t sample_shot_capacity();
sv_status launch_tile_pass(sv_state *s, const TilePass &p, int batch);
// Append a complex64 dense matrix of k <= 3 qubits (row-major U) to a pool
// in the row-pair layout the packed tile ops read: for p < 2^k / 2 and
// column y, (Re U[2p][y], Re U[2p+1][y]) then (Im U[2p][y], Im U[2p+1][y]).
void put_pairs_c64(std::vector<uint8_t> &pool, const cd *U, int k);
// perm[c] = row of the single 1 in column c when U (2^k x 2^k, k <= 5) is a 0/1 permutation matrix
bool permutation_of(const std::vector<cd> &U, int k, int *perm);
// host copy of a pass's ops (the pass's first op) and of the program's matrix pool
struct HostPass {
  const TileOp *ops;
  const uint8_t *mats;
};
sv_status launch_tile_pass_on(sv_state *s, const TilePass &p, int batch, cudaStream_t stream,
                              const HostPass *host = nullptr);
sv_status launch_tile_tc(sv_state *s, const TilePass &p, cudaStream_t stream);   // k_tile_tc.cu
// pipelined split-BF16 tile pass (k_tile_tcp.cu): at most kTcpMaxBlocks
// tensor-core blocks per pass, whose B operands stay in shared memory
constexpr int kTcpMaxBlocks = 6;
sv_status launch_tile_tcp(sv_state *s, const TilePass &p, const HostPass &host, cudaStream_t stream);
// a pass the pipelined kernel runs: 12-qubit tiles, 1..kTcpMaxBlocks ops, all 5-qubit TOP_TC
bool tcp_pass_ok(const TilePass &p, const HostPass &host);
// The pipelined kernel gives block j of a pass its own shared-memory layout:
// tile bits 0 and pair_bit swapped, where pair_bit is 0 for the first block
// (and for the tile store after the last) and the block's first target
// op.t[0] for the others, so that those blocks gather member pairs (y, y+1)
// as 16-byte units, and a block whose first target is the next layout's
// pair bit scatters them the same way.
inline int tcp_pair_bit(const TileOp *ops, int nops, int j) {
  return (j <= 0 || j >= nops) ? 0 : (int)ops[j].t[0];
}
// plan-time row map of a TOP_TC op for the pipelined kernel's bank layout,
// for a block gathered under the layout with pair bit pair_gather and
// scattered under the one with pair bit pair_scatter
void tcp_row_positions(TileOp &op, int pair_gather, int pair_scatter);
// host replay of a pipelined pass's shared-memory addressing; "" when sound
std::string tcp_layout_selftest(const TilePass &p, const HostPass &host, int *pair_gathers = nullptr,
                                int *pair_scatters = nullptr);
// tensor-core 5-qubit block (k_tc.cu)
size_t tc_matrix_words(sv_prec mode, int k);
void tc_pack_matrix(const std::vector<cd> &U, sv_prec mode, std::vector<uint32_t> &out);
sv_status launch_dense_tc(sv_state *s, void *amps, const int *targets, const uint32_t *bmat_dev, sv_prec mode,
                          uint64_t spin_limit, cudaStream_t stream);
// a 6-qubit dense block on the tensor cores, split-BF16, a pass of its own (k_tc.cu)
sv_status launch_dense_tc6(sv_state *s, void *amps, const int *targets, const uint32_t *bmat_dev,
                           uint64_t spin_limit, cudaStream_t stream);
// one pass of a program (tile pass or tensor-core block) on stream st
sv_status launch_any_pass(sv_state *s, const TilePass &tp, int batch, cudaStream_t st,
                          const HostPass *host = nullptr);
sv_status launch_tile_persist(sv_state *s, const PersistArgs &A, int m_max, int *grid_out, cudaStream_t st);
sv_status launch_wait_selftest(cudaStream_t st, const uint32_t *never, uint32_t *err, uint64_t limit);
int tile_threads(int m, sv_dtype dt);
size_t tile_smem(sv_dtype dt, int m, int nvec);

}  // namespace sv
