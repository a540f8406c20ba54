// Host-side launchers of the IG kernels, called by the C ABI layer
// (ig_capi.cu).  Internal row arrays use a padded stride of KT words,
// KT = the smallest of {1, 2, 4, 8, 16} >= K; the padding words are zero.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <new>
#include <vector>

#include "../../include/ig.h"

namespace igk {

// The status of an entry point whose body threw (no C++ exception may cross
// the C ABI): IG_E_NOMEM for a failed host allocation, IG_E_INTERNAL for any
// other exception; the message names the entry point.
int report_exception(const char* where, bool out_of_memory) noexcept;

// Runs the body of an exported entry point, or work that one hands to a
// helper thread, so that an exception becomes a status instead of ending the
// caller's process.
template <class Body>
int guarded(const char* where, Body&& body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return report_exception(where, true);
  } catch (...) {
    return report_exception(where, false);
  }
}

// Rows of every internally staged row array are allocated in multiples of
// this many rows, so that whole TMA tiles can always be copied in bounds.
constexpr int64_t kRowPad = 256;

inline int padded_words(int K) {
  int kt = 1;
  while (kt < K) kt *= 2;
  return kt;
}

inline int64_t pad_rows(int64_t n) { return ((n + kRowPad - 1) / kRowPad) * kRowPad; }

int num_sms();

// Device pointers.  device_of: true if p is CUDA device (or managed) memory,
// with *dev set to the device that owns it.  is_device_pointer: the same
// test, and the calling thread's current device is switched to the owner,
// so that the rest of the call allocates and launches there; entry points
// that call it hold a DeviceRestore, which puts the caller's device back
// when the call returns.
bool device_of(const void* p, int* dev);
bool is_device_pointer(const void* p);
struct DeviceRestore {
  int dev = -1;
  DeviceRestore() {
    if (cudaGetDevice(&dev) != cudaSuccess) {
      cudaGetLastError();
      dev = -1;
    }
  }
  ~DeviceRestore() {
    int cur = -1;
    if (dev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != dev) cudaSetDevice(dev);
  }
  DeviceRestore(const DeviceRestore&) = delete;
  DeviceRestore& operator=(const DeviceRestore&) = delete;
};

// Stage timing (ig_prof_*): prof_begin records a CUDA event on s when timing
// is on and returns a token (nullptr otherwise); prof_end records the
// closing event and files the pair under the stage.
void* prof_begin(int stage, cudaStream_t s);
void prof_end(void* token);
// Adds executed subset tests to a stage's tally (while timing is on).
void prof_add_work(int stage, int64_t tests);
constexpr int kStageIndexBuild = 19;

// Adds n to the library's count of kernel launches (ig_launch_count).
void count_launches(int n);

// probe.cu: one throughput probe (ig_probe).
int probe_run(int probe, int arg, double* rate, double* ms, double* cycles);

// Read-only view of a fitted model's device arrays (for entry points defined
// outside ig_capi.cu).
struct ModelView {
  int K, KT;
  const uint64_t* words_kt[2];  // stride KT, pad_rows rows
  const uint64_t* score[2];     // pad_rows entries
  int64_t n_pat[2];
  int reg3;
  double thr;
};
}  // namespace igk
struct ig_model;
namespace igk {
void model_view(const ig_model* m, ModelView* v);

// Records msg as the calling thread's last error and returns code.
int report_error(int code, const char* msg);

// ---- encode.cu --------------------------------------------------------------
// Eq. 5 one-hot packing; offsets[f] = sum of cards before f (device array).
cudaError_t launch_encode(const uint16_t* codes, int64_t n, int F,
                          const uint32_t* offsets, const uint16_t* cards,
                          uint64_t* out, int K, int* status, cudaStream_t s);

// Exclusive scan of cnt[0..len) into off[0..len] (off[len] = total), one
// block (prune.cu).
cudaError_t launch_small_scan(const uint32_t* cnt, int len, uint32_t* off, cudaStream_t s);

// Stable split of rows (stride K) by label into class arrays (stride KT):
// normal rows to x0, attack rows to x1.  counts[0..1] receive the sizes.
cudaError_t launch_split(const uint64_t* rows, const uint8_t* labels, int64_t n,
                         int K, int KT, uint64_t* x0, uint64_t* x1,
                         unsigned long long* counts, int* status, cudaStream_t s);

// ---- dedup.cu -----------------------------------------------------------------
// Hash set of candidate itemsets keyed by the pair (i, j) whose intersection
// they are (see dedup.cu for the slot format).
struct PairTable {
  uint64_t* slots = nullptr;                // cap words, 0 = empty
  uint64_t mask = 0;                        // cap - 1, cap a power of two
  unsigned long long* count = nullptr;      // keys stored (added per warp every `flush` keys
                                            // and when its CTA ends)
  unsigned long long limit = 0;             // pair tiles stop once count >= limit
  uint64_t max_probe = 0;                   // slots one insert may probe before it fails
  int* failed_band = nullptr;               // lowest band that ran out of room
  uint32_t flush = 0;                       // set by launch_pair_insert
};

constexpr int kPairTile = 64;  // records per side of a pair tile (one band = one tile row)

// Inserts x_i AND x_j for every i <= j (i == j gives the record itself),
// skipping empty intersections, for every pair tile in bands >= band_lo of
// the upper triangle; one launch.
// flag[i] = 1 for every row of X[0, n) (stride KT) whose content an
// earlier-claimed row already has, 0 for one row per distinct content.
// table: cap uint32 slots (cap a power of two above n), all 0xffffffff.
cudaError_t launch_mark_repeats(const uint64_t* X, int64_t n, int KT, uint32_t* table,
                                uint64_t cap, uint32_t* flag, cudaStream_t s);
// n_dev (optional): the number of rows on the device, at most n (n then
// sizes the grid only).
cudaError_t launch_pair_insert(const uint64_t* X, int64_t n, int KT, int64_t band_lo,
                               PairTable t, int* status, cudaStream_t s,
                               const unsigned long long* n_dev = nullptr);
// One table of a multi-table pair launch: the records X[0, n) (KT words
// per row), the bands [band_lo, ceil(n / kPairTile)) and the table (its
// flush set by the caller, see pair_multi_grid_warps).
struct PairJob {
  const uint64_t* X = nullptr;
  int64_t n = 0;
  int64_t band_lo = 0;
  int KT = 0;
  PairTable t;
};
// The pair tiles of every job, of any word counts, in one launch of a
// persistent grid drawing tiles from a device-side queue: tile_off[j]
// (device, n_jobs + 1 entries) numbers job j's tiles band by band;
// next_tile (device) must start at 0.
cudaError_t launch_pair_insert_multi(const PairJob* jobs, int n_jobs, const int64_t* tile_off,
                                     unsigned long long* next_tile, int* status, cudaStream_t s);
// Warps of the multi-table launch's grid (for the jobs' flush intervals).
int pair_multi_grid_warps();
// Re-inserts every key of the table `from` (from_cap slots) into `to`.
cudaError_t launch_rehash(const uint64_t* X, const uint64_t* from, uint64_t from_cap,
                          PairTable to, int KT, int* status, cudaStream_t s);
// Appends every stored key (recomputed from its pair) to out (stride KT,
// room for out_rows keys; a key beyond them is not written and sets
// ST_COUNT); out_count must start at 0.
cudaError_t launch_compact(const uint64_t* X, const uint64_t* slots, uint64_t cap, int KT,
                           uint64_t* out, int64_t out_rows, unsigned long long* out_count,
                           int* status, cudaStream_t s);

// ---- subset.cu --------------------------------------------------------------
enum SubsetMode { MODE_ANY = 0, MODE_COUNT = 1, MODE_SUM = 2 };

// MODE_ANY:   flag[i] = 1 if own row i is contained in some stream row.
// MODE_COUNT: cnt[i] += number of stream rows containing own row i.
// MODE_SUM:   sum[i] += sum of score[j] over stream rows j contained in own
//             row i.
// own: n_own rows of stride own_stride (any K <= KT, extra words read as 0).
// stream: n_stream rows of stride KT, allocated to pad_rows(n_stream) rows.
struct SubsetArgs {
  int mode;
  int KT;
  const uint64_t* own;
  int64_t n_own;
  int own_stride;
  const uint64_t* stream;
  const uint64_t* stream_score;  // MODE_SUM only, padded like stream
  int64_t n_stream;
  uint32_t* out_u32;             // ANY / COUNT
  unsigned long long* out_u64;   // SUM
  int* status;
  // Optional: the number of own rows, read on the device (n_own is then
  // only an upper bound used to size the grid).
  const unsigned long long* n_own_dev = nullptr;
};
cudaError_t launch_subset(const SubsetArgs& a, cudaStream_t s);

// ---- subset_tc.cu (tensor-core form of the subset tests) --------------------
// Operand images: rows expanded to one FP8 byte per item in the shared-memory
// layout of the MMA, in tiles of 128 rows.  own_side images feed the M side
// (one tile per CTA), the others the streamed N side.  `complement` images
// hold NOT(row) (used for the records being tested against).
bool tc_supported(int KT);
size_t tc_image_bytes(int64_t n, int KT, bool own_side);
cudaError_t launch_expand(const uint64_t* rows, int64_t n, int stride, int KT, bool complement,
                          bool own_side, uint8_t* img, cudaStream_t s);
// One block of work for the tensor-core kernel on the item index: the
// resident rows own_first .. own_first + own_count - 1 (at most 128) of a
// group against its streamed rows str_first .. str_first + str_count - 1, in
// b_tiles tiles of 128 rows (grouped row numbers).
struct TcItem {
  int64_t own_first, str_first;
  int32_t own_count, b_tiles, str_count, pad;
};

struct TcArgs {
  int mode;
  int KT;
  const uint8_t* a_img;                 // own image (patterns, or complemented records for SUM)
  int64_t n_own;                        // own rows (upper bound when n_own_dev is given)
  const unsigned long long* n_own_dev;  // optional device-side own count
  const uint8_t* b_img;                 // stream image
  int64_t b_tile0;                      // first 128-row stream tile to use
  int64_t n_stream;                     // stream rows from tile b_tile0 on
  const uint64_t* score;                // MODE_SUM: S per stream row (from b_tile0 * 128)
  uint32_t* out_u32;
  unsigned long long* out_u64;
  int* status;
};
cudaError_t launch_subset_tc(const TcArgs& a, cudaStream_t s);

// ---- prune.cu (subset tests restricted by an item index) --------------------
struct WorkItem {
  int64_t own_begin, own_count, str_begin, str_count;
  int32_t own_keyed;  // 1: registers hold patterns (keyed rows), 0: records
  int32_t q;          // own rows per thread (1, 2 or 4); 256 * q rows per block
};
struct GroupedArgs {
  int mode;
  int KT;
  const WorkItem* items;
  int64_t n_items;
  const uint64_t* keyed;
  const uint32_t* keyed_ids;
  const uint64_t* keyed_score;
  const uint64_t* multi;
  const uint32_t* multi_ids;
  uint32_t* out_u32;
  unsigned long long* out_u64;
  int* status;
};
cudaError_t launch_grouped_subset(const GroupedArgs& a, cudaStream_t s);

// Record index ("multi" side): every record filed under each item it
// holds, with the item counts.  Built once, used by any number of indexed
// subset tests.  Not built (usable = false) when the records fill more than
// max_fill of all item slots: then nearly every group holds nearly every
// record and the dense kernels are faster.  Synchronizes the stream.
struct RecordIndex {
  int K = 0, KT = 0, L = 0;
  int64_t n_rows = 0, n_copies = 0;
  bool usable = false;
  uint64_t* rows = nullptr;   // grouped copies, stride KT (+256 rows of padding)
  uint32_t* ids = nullptr;    // original record of each copy
  uint32_t* small = nullptr;  // freq[L] | off[L+1] | cursor[L]
  uint32_t* freq = nullptr;
  uint32_t* off = nullptr;
  std::vector<uint32_t> h_off;
};
// id_map (optional, n entries): the id filed for row i is id_map[i] instead
// of i (rows given in another order than the caller's).
cudaError_t build_record_index(const uint64_t* rows, int64_t n, int stride, int K, int KT,
                               double max_fill, RecordIndex* idx, cudaStream_t s,
                               const uint32_t* id_map = nullptr);
void release_record_index(RecordIndex* idx, cudaStream_t s);

// A subset test of "keyed" rows (patterns: MODE_ANY / MODE_COUNT own rows,
// MODE_SUM stream rows) against the records of an index, restricted to the
// pairs that share the pattern's key item (its item held by the fewest
// records).  Outputs are indexed like the dense kernels': by pattern for
// ANY / COUNT, by record for SUM.  Requires KT >= 2.  Synchronizes the
// stream once.
struct IndexedArgs {
  int mode;
  const RecordIndex* index;
  const uint64_t* keyed;
  int64_t n_keyed;
  int keyed_stride;
  const uint64_t* keyed_score;  // MODE_SUM: S of each keyed row
  uint32_t* out_u32;
  unsigned long long* out_u64;
  int* status;
  int64_t* tests_out;   // subset tests executed (tensor-core form: pinned host memory,
                        // written when the stream gets there)
  int prof_stage = -1;  // stage under which the grouped kernel is timed
  int max_q = 4;        // most own rows per thread of a block (1, 2, 4)
  int flip_factor = 2;  // side ratio before the non-result side goes to registers
  int tc = 0;           // run the blocks on the tensor cores (KT 2, 4, 8)
  // Optional: the keyed row count on the device; n_keyed is then its upper
  // bound (no host read-back is needed before the index is built).
  const unsigned long long* n_keyed_dev = nullptr;
  uint64_t score_max = ~uint64_t(0);  // MODE_SUM: an upper bound of keyed_score
};
cudaError_t indexed_subset(const IndexedArgs& a, cudaStream_t s);

// The pattern side of the item index, built once and reusable: patterns
// filed under their key item (the item with the smallest `freq`; group L
// holds patterns with an item of freq 0).  Synchronizes the stream once to
// read the group offsets back, unless built without host offsets.
struct KeyedIndex {
  int K = 0, KT = 0, L = 0;
  int64_t n = 0;
  uint64_t* rows = nullptr;   // grouped patterns, stride KT (+256 rows of padding)
  uint32_t* ids = nullptr;    // original pattern of each grouped row
  uint64_t* score = nullptr;  // S of each grouped pattern (when built with scores)
  uint32_t* off = nullptr;    // group offsets, L + 2 entries
  std::vector<uint32_t> h_off;
};
// n_dev (optional): the number of rows on the device, at most n (an upper
// bound then, used for sizes); out->n is the number filed.  With
// host_offsets false nothing is read back and the stream is not
// synchronized: h_off stays empty and out->n is the bound n (for the
// tensor-core form, which builds its work items on the device).
cudaError_t build_keyed_index(const uint64_t* keyed, int64_t n, int stride, int K, int KT,
                              const uint32_t* freq, const uint64_t* score, KeyedIndex* out,
                              cudaStream_t s, const unsigned long long* n_dev = nullptr,
                              bool host_offsets = true);
void release_keyed_index(KeyedIndex* k, cudaStream_t s);
// The item-index test with its blocks run on the tensor cores (KT 2, 4, 8):
// the patterns go to resident tiles, the records stream; packed rows are
// expanded to operand tiles by a persistent kernel whose work items are
// built on the device from the indexes' device offsets (the keyed indexes
// need no host offsets).  Same results as the integer grouped kernel.
// tests_out (optional) must be pinned host memory: the executed tests are
// copied there when the stream reaches this point (valid after the caller's
// next synchronization).
// score_max (MODE_SUM): an upper bound of the keyed rows' scores; below
// 2^27 the kernel sums each hit column's scores over a warp in 32 bits
// before adding them to the record.
//
// indexed_subset_tc_classes: the same for n_cls keyed indexes (1, or 2 with
// MODE_SUM: both classes' patterns against one record index in one launch,
// class c's sums into out_sum[c]); tests_out and score_max have n_cls entries.
cudaError_t indexed_subset_tc_classes(int mode, const RecordIndex& idx, const KeyedIndex* const* kx,
                                      int n_cls, uint32_t* out_u32,
                                      unsigned long long* const* out_sum, int* status,
                                      int64_t* tests_out, int prof_stage,
                                      const uint64_t* score_max, cudaStream_t s);
cudaError_t indexed_subset_tc(int mode, const RecordIndex& idx, const KeyedIndex& kx,
                              uint32_t* out_u32, unsigned long long* out_u64, int* status,
                              int64_t* tests_out, int prof_stage, uint64_t score_max,
                              cudaStream_t s);
// indexed_subset with a prebuilt pattern side; no synchronization.  The
// tensor-core form writes *tests_out asynchronously (pinned host memory,
// valid after the caller's next synchronization), the integer form at once.
cudaError_t indexed_subset_prebuilt(int mode, const RecordIndex& idx, const KeyedIndex& kx,
                                    uint32_t* out_u32, unsigned long long* out_u64, int* status,
                                    int64_t* tests_out, int prof_stage, int max_q,
                                    int flip_factor, int tc, cudaStream_t s,
                                    uint64_t score_max = ~uint64_t(0));
// freq[l] += number of the n rows holding item l (rows of stride `stride`, K words).
cudaError_t launch_item_histogram(const uint64_t* rows, int64_t n, int stride, int K, int L,
                                  uint32_t* freq, cudaStream_t s);

// Keeps the rows whose flag is zero: out gets them (stride KT), out_count
// the number kept (must start at 0).  With n_dev given, the row count is
// read on the device and n is only an upper bound.
cudaError_t launch_select_unflagged(const uint64_t* rows, int64_t n, int KT,
                                    const uint32_t* flag, uint64_t* out,
                                    unsigned long long* out_count, cudaStream_t s,
                                    const unsigned long long* n_dev = nullptr);

// S = f * popcount(row)^2 (Eq. 2); smax (optional, must start at 0)
// receives the largest S.
cudaError_t launch_pattern_score(const uint64_t* rows, int64_t n, int KT,
                                 const uint32_t* f, uint64_t* S, cudaStream_t s,
                                 unsigned long long* smax = nullptr);

// Regulations 1-3 -> label (1 attack).
cudaError_t launch_labels(const unsigned long long* A, const unsigned long long* N,
                          int64_t m, int reg3, double threshold, uint8_t* out,
                          cudaStream_t s);

// ---- sort.cu ----------------------------------------------------------------
// Canonical order of n keys (stride KT): ascending as KT-word unsigned
// integers, word KT-1 most significant; equal keys may repeat.  keys_out (n
// rows) receives the sorted rows and must not overlap keys; `work` is
// unused (the sort allocates its own 40 bytes per key).  perm_out (optional,
// n entries): the input row of each sorted row.
cudaError_t canonical_sort(const uint64_t* keys, int64_t n, int KT, uint64_t* keys_out,
                           uint64_t* work, cudaStream_t s, uint32_t* perm_out = nullptr);

// payload_sorted[pos of keys[i] in sorted] = payload[i] (binary search;
// ST_BAD_INPUT if a key is missing).  sorted and keys: n rows, stride KT.
cudaError_t launch_place_payload(const uint64_t* sorted, int64_t n, int KT, const uint64_t* keys,
                                 const uint32_t* payload, uint32_t* payload_sorted, int* status,
                                 cudaStream_t s);
// ST_BAD_INPUT if a sorted list holds an empty row or a repeated row.
cudaError_t launch_check_strict(const uint64_t* sorted, int64_t n, int KT, int* status,
                                cudaStream_t s);

}  // namespace igk
