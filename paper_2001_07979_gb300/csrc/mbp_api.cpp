// C ABI of libmbp: argument validation, code upload and the entry points
// declared in include/mbp.h. Kernels and the decode driver are in mbp_kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mbp_nbp.h"

namespace mbp {

static thread_local std::string g_err;

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_error(cudaError_t e, const char* what) {
  return set_error(MBP_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// Device or managed memory that the current device's kernels may address: device memory must belong to the
// current device (the kernels of a decode run there); managed memory migrates on access.
static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  if (a.type != cudaMemoryTypeDevice) return false;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.device == cur;
}

// The device that is current for this host thread, or -1.
static int current_device() {
  int d = -1;
  if (cudaGetDevice(&d) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return d;
}

// ---- kernel accounting (mbp_profile_*)
namespace {
struct Prof {
  struct Pending {
    int family, kernels;
    cudaEvent_t a, b;
  };
  bool on = false;
  int64_t launches[MBP_KERNEL_FAMILIES] = {};
  double ms[MBP_KERNEL_FAMILIES] = {};
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t open = nullptr;
  cudaEvent_t take() {
    if (pool.empty()) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      return e;
    }
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  void drain() {
    for (auto& p : pending) {
      float t = 0.f;
      if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
        ms[p.family] += t;
        launches[p.family] += p.kernels;
      }
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
};
thread_local Prof g_prof;
}  // namespace

void prof_enable(bool on) {
  g_prof.drain();
  for (int k = 0; k < MBP_KERNEL_FAMILIES; ++k) {
    g_prof.launches[k] = 0;
    g_prof.ms[k] = 0.0;
  }
  g_prof.on = on;
}

bool prof_on() { return g_prof.on; }

void prof_begin(int, cudaStream_t s) {
  if (!g_prof.on) return;
  g_prof.open = g_prof.take();
  if (g_prof.open) cudaEventRecord(g_prof.open, s);
}

void prof_end(int family, cudaStream_t s, int kernels) {
  if (!g_prof.on || !g_prof.open) return;
  cudaEvent_t e = g_prof.take();
  if (!e) return;
  cudaEventRecord(e, s);
  g_prof.pending.push_back({family, kernels, g_prof.open, e});
  g_prof.open = nullptr;
  if (g_prof.pending.size() > 512) g_prof.drain();
}

int prof_get(int family, int64_t* launches, double* ms) {
  if (family < 0 || family >= MBP_KERNEL_FAMILIES) return set_error(MBP_EINVAL, "unknown kernel family %d", family);
  g_prof.drain();
  if (launches) *launches = g_prof.launches[family];
  if (ms) *ms = g_prof.ms[family];
  return MBP_OK;
}

}  // namespace mbp

using namespace mbp;

namespace {

#define REQUIRE(cond, ...)                         \
  do {                                             \
    if (!(cond)) return set_error(MBP_EINVAL, __VA_ARGS__); \
  } while (0)

#define REQUIRE_DEV(p, name) \
  REQUIRE(is_device_ptr(p), "%s must be a device pointer of the current device", name)

#define REQUIRE_CODES_HERE(c)                                                                              \
  REQUIRE((c)->device == current_device(), "codes were uploaded to device %d, but device %d is current", \
          (c)->device, current_device())

// MBP_SCHED_AUTO takes the graph schedule wherever it runs the options (flooding sum-product, FP32, FP16 or
// BF16 storage, floating-point accumulation), else the streaming schedule.
bool graph_schedule(const mbp_opts* o) {
  if (o->schedule == MBP_SCHED_GRAPH) return true;
  return o->schedule == MBP_SCHED_AUTO && o->rule == MBP_RULE_SUM_PRODUCT && o->update == MBP_UPDATE_FLOODING &&
         o->msg_dtype != MBP_MSG_F64 && o->accumulate != MBP_ACC_FIXED;
}

int validate_opts(const mbp_opts* o) {
  REQUIRE(o, "opts is NULL");
  REQUIRE(o->msg_dtype == MBP_MSG_F32 || o->msg_dtype == MBP_MSG_F64 || o->msg_dtype == MBP_MSG_F16 ||
              o->msg_dtype == MBP_MSG_BF16,
          "unknown msg_dtype %d", o->msg_dtype);
  REQUIRE(o->early_exit == 0 || o->early_exit == 1, "early_exit must be 0 or 1");
  REQUIRE(std::isfinite(o->l_max) && o->l_max > 0, "l_max must be finite and > 0");
  REQUIRE(o->accumulate == MBP_ACC_AUTO || o->accumulate == MBP_ACC_FLOAT || o->accumulate == MBP_ACC_FIXED,
          "unknown accumulate mode %d", o->accumulate);
  REQUIRE(o->schedule == MBP_SCHED_AUTO || o->schedule == MBP_SCHED_STREAMING || o->schedule == MBP_SCHED_RESIDENT ||
              o->schedule == MBP_SCHED_GRAPH,
          "unknown schedule %d", o->schedule);
  REQUIRE(o->rule == MBP_RULE_SUM_PRODUCT || o->rule == MBP_RULE_MIN_SUM, "unknown check rule %d", o->rule);
  REQUIRE(o->update == MBP_UPDATE_FLOODING || o->update == MBP_UPDATE_MATRIX_SERIAL, "unknown update order %d",
          o->update);
  if (o->rule != MBP_RULE_SUM_PRODUCT || o->update != MBP_UPDATE_FLOODING) {
    if (o->schedule != MBP_SCHED_AUTO && o->schedule != MBP_SCHED_STREAMING)
      return set_error(MBP_EUNSUPPORTED, "the min-sum rule and the matrix-serial order run the streaming schedule");
    if (o->accumulate == MBP_ACC_FIXED)
      return set_error(MBP_EUNSUPPORTED, "the min-sum rule and the matrix-serial order accumulate in floating point");
    if (o->rule == MBP_RULE_MIN_SUM && o->msg_dtype == MBP_MSG_F64)
      return set_error(MBP_EUNSUPPORTED, "the min-sum rule runs with FP32, FP16 or BF16 messages");
  }
  if (o->schedule == MBP_SCHED_GRAPH) return multi_check_opts(o);
  return MBP_OK;
}

// The single group of a single-code decode under MBP_SCHED_GRAPH (pointers filled in by the caller).
mbp_group one_group(const mbp_codes* c, int F) {
  mbp_group g;
  std::memset(&g, 0, sizeof g);
  g.codes = c;
  g.F = F;
  return g;
}

int single_workspace(const mbp_codes* c, int F, const mbp_opts* o, bool host_io, size_t* need) {
  if (!graph_schedule(o)) {
    *need = workspace_bytes(c->d, F, o->msg_dtype, host_io);
    return MBP_OK;
  }
  const mbp_group g = one_group(c, F);
  return multi_workspace(&g, 1, o, host_io, need);
}

// The decoder state of a single-code decode inside its workspace.
int single_state(const mbp_codes* c, int F, const mbp_opts* o, bool host_io, void* ws, DevState* st) {
  if (!graph_schedule(o)) {
    carve_workspace(c->d, F, o->msg_dtype, host_io, ws, st);
    return MBP_OK;
  }
  const mbp_group g = one_group(c, F);
  mbp_opts oo = *o;
  oo.workspace = ws;
  return multi_group_state(&g, 1, 0, &oo, host_io, st);
}

int check_workspace(const mbp_codes* c, int F, const mbp_opts* o) {
  size_t need = 0;
  int rc = single_workspace(c, F, o, o->host_io != 0, &need);
  if (rc) return rc;
  REQUIRE(o->workspace, "opts->workspace is NULL (size it with mbp_decode_workspace_size)");
  REQUIRE((reinterpret_cast<uintptr_t>(o->workspace) & 255) == 0, "workspace must be 256-byte aligned");
  REQUIRE(o->workspace_bytes >= need, "workspace too small: %zu bytes given, %zu needed", o->workspace_bytes, need);
  REQUIRE_DEV(o->workspace, "workspace");
  return MBP_OK;
}

int common_decode_checks(const mbp_codes* codes, int F, int max_iter, const mbp_opts* opts) {
  REQUIRE(codes, "codes is NULL");
  REQUIRE(F >= 0, "F must be >= 0");
  REQUIRE(max_iter >= 0 && max_iter <= 1000000, "max_iter must be in [0, 1e6]");
  if (F == 0) return MBP_OK;
  REQUIRE_CODES_HERE(codes);
  int rc = validate_opts(opts);
  if (rc) return rc;
  return check_workspace(codes, F, opts);
}

}  // namespace

extern "C" {

void mbp_default_opts(mbp_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->msg_dtype = MBP_MSG_F32;
  o->early_exit = 1;
  o->l_max = 20.0;
}

const char* mbp_last_error_string(void) { return g_err.c_str(); }

int mbp_version(void) { return 100; }

int mbp_create_codes(const mbp_csr* H, int u, mbp_codes** out) {
  g_err.clear();
  REQUIRE(out, "out is NULL");
  *out = nullptr;
  REQUIRE(H, "H is NULL");
  REQUIRE(u >= 1, "u must be >= 1");
  if (u > kMaxU) return set_error(MBP_EUNSUPPORTED, "u = %d exceeds the limit of %d matrices", u, kMaxU);
  const int32_t n = H[0].n;
  REQUIRE(n > 0, "n must be > 0");
  int64_t m_tot = 0, e_tot = 0;
  for (int l = 0; l < u; ++l) {
    const mbp_csr& h = H[l];
    REQUIRE(h.n == n, "matrix %d has n = %d, matrix 0 has n = %d", l, h.n, n);
    REQUIRE(h.m >= 0 && h.nnz >= 0, "matrix %d: negative m or nnz", l);
    REQUIRE(h.row_ptr, "matrix %d: row_ptr is NULL", l);
    REQUIRE(h.nnz == 0 || h.col_idx, "matrix %d: col_idx is NULL", l);
    REQUIRE(h.row_ptr[0] == 0, "matrix %d: row_ptr[0] != 0", l);
    for (int32_t j = 0; j < h.m; ++j)
      REQUIRE(h.row_ptr[j + 1] >= h.row_ptr[j], "matrix %d: row_ptr decreases at row %d", l, j);
    REQUIRE(h.row_ptr[h.m] == h.nnz, "matrix %d: row_ptr[m] = %d != nnz = %d", l, h.row_ptr[h.m], h.nnz);
    std::vector<int32_t> row;
    for (int32_t j = 0; j < h.m; ++j) {
      const int32_t d = h.row_ptr[j + 1] - h.row_ptr[j];
      if (d > kMaxRowDeg)
        return set_error(MBP_EUNSUPPORTED, "matrix %d row %d has %d edges; the limit is %d", l, j, d, kMaxRowDeg);
      row.assign(h.col_idx + h.row_ptr[j], h.col_idx + h.row_ptr[j + 1]);
      for (int32_t c : row) REQUIRE(c >= 0 && c < n, "matrix %d row %d: column %d outside [0, %d)", l, j, c, n);
      std::sort(row.begin(), row.end());
      REQUIRE(std::adjacent_find(row.begin(), row.end()) == row.end(), "matrix %d row %d repeats a column", l, j);
    }
    m_tot += h.m;
    e_tot += h.nnz;
  }
  REQUIRE(m_tot <= INT32_MAX / 2 && e_tot <= INT32_MAX / 2, "code too large");

  // ---- host layout
  DevCode d{};
  d.n = n;
  d.u = u;
  d.m_tot = static_cast<int32_t>(m_tot);
  d.e_tot = e_tot;
  d.row_first[0] = 0;
  for (int l = 0; l < u; ++l) {
    d.m[l] = H[l].m;
    d.row_first[l + 1] = d.row_first[l] + H[l].m;
  }
  std::vector<int32_t> row_ptr(m_tot + 1), col_idx(std::max<int64_t>(e_tot, 1)), row_deg(m_tot);
  std::vector<uint8_t> row_mat(std::max<int64_t>(m_tot, 1));
  {
    int64_t e = 0, r = 0;
    row_ptr[0] = 0;
    for (int l = 0; l < u; ++l)
      for (int32_t j = 0; j < H[l].m; ++j, ++r) {
        for (int32_t k = H[l].row_ptr[j]; k < H[l].row_ptr[j + 1]; ++k) col_idx[e++] = H[l].col_idx[k];
        row_ptr[r + 1] = static_cast<int32_t>(e);
        row_deg[r] = row_ptr[r + 1] - row_ptr[r];
        row_mat[r] = static_cast<uint8_t>(l);
      }
  }
  int32_t max_deg = 0, min_deg = 0;
  for (int64_t r = 0; r < m_tot; ++r) {
    max_deg = std::max(max_deg, row_deg[r]);
    if (row_deg[r] > 0) min_deg = min_deg == 0 ? row_deg[r] : std::min(min_deg, row_deg[r]);
  }
  d.max_row_deg = max_deg;
  d.min_row_deg = min_deg > 0 ? min_deg : 1;
  // The decoder visits the stacked rows matrix by matrix, each matrix's rows in
  // degree order (ties keep the stacked order): row position p owns the slots
  // slice_base[p] .. slice_base[p+1] - 1, and matrix l's rows are the positions
  // row_pos[l] .. row_pos[l+1] - 1 (the matrix-serial schedule's steps).
  // The order is internal: syndrome bits are looked up through perm_mat /
  // perm_local, and C2V exports go through edge_slot.
  std::vector<int32_t> order(m_tot);
  for (int64_t p = 0; p < m_tot; ++p) order[p] = static_cast<int32_t>(p);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return row_mat[a] != row_mat[b] ? row_mat[a] < row_mat[b] : row_deg[a] < row_deg[b];
  });
  for (int l = 0; l <= u; ++l) d.row_pos[l] = d.row_first[l];  // matrices stay in stacked order
  std::vector<uint8_t> perm_mat(std::max<int64_t>(m_tot, 1));
  std::vector<int32_t> perm_local(std::max<int64_t>(m_tot, 1)), row_at(std::max<int64_t>(m_tot, 1));
  std::vector<int32_t> slice_base(m_tot + 1);
  slice_base[0] = 0;
  for (int64_t p = 0; p < m_tot; ++p) {
    const int32_t r = order[p];
    perm_mat[p] = row_mat[r];
    perm_local[p] = r - d.row_first[row_mat[r]];
    row_at[r] = int32_t(p);
    slice_base[p + 1] = slice_base[p] + row_deg[r];
  }
  d.s_tot = slice_base[m_tot];
  std::vector<int32_t> slot_col(std::max<int64_t>(d.s_tot, 1), -1), edge_slot(std::max<int64_t>(e_tot, 1));
  for (int64_t p = 0; p < m_tot; ++p) {
    const int32_t r = order[p];
    for (int32_t k = 0; k < row_deg[r]; ++k) {
      const int32_t slot = slice_base[p] + k;
      slot_col[slot] = col_idx[row_ptr[r] + k];
      edge_slot[row_ptr[r] + k] = slot;
    }
  }
  std::vector<int32_t> col_ptr(n + 1, 0), col_slot(std::max<int64_t>(e_tot, 1));
  for (int64_t e = 0; e < e_tot; ++e) col_ptr[col_idx[e] + 1]++;
  int32_t max_cdeg = 0;
  for (int32_t i = 0; i < n; ++i) max_cdeg = std::max(max_cdeg, col_ptr[i + 1]);
  if (max_cdeg > kMaxColDeg)
    return set_error(MBP_EUNSUPPORTED, "a variable node has %d edges over all matrices; the limit is %d", max_cdeg,
                     kMaxColDeg);
  d.max_col_deg = max_cdeg;
  for (int32_t i = 0; i < n; ++i) col_ptr[i + 1] += col_ptr[i];
  {
    std::vector<int32_t> fill(col_ptr.begin(), col_ptr.end() - 1);
    for (int64_t e = 0; e < e_tot; ++e) col_slot[fill[col_idx[e]]++] = edge_slot[e];  // stacked-row order
  }
  // variable nodes by degree class, each with a dense table of its slots (the variable-node kernel then
  // loads a node and its slots together)
  std::vector<int32_t> vnode(n), vslot(std::max<int64_t>(e_tot, 1)), vrow(std::max<int64_t>(e_tot, 1));
  std::vector<int32_t> slot_row(std::max<int64_t>(d.s_tot, 1));
  for (int64_t p = 0; p < m_tot; ++p)  // row position << 6 | degree - 1 (degree <= kMaxRowDeg = 64)
    for (int32_t q = slice_base[p]; q < slice_base[p + 1]; ++q)
      slot_row[q] = int32_t(p << 6) | (slice_base[p + 1] - slice_base[p] - 1);
  for (int32_t i = 0; i < n; ++i) vnode[i] = i;
  std::stable_sort(vnode.begin(), vnode.end(), [&](int32_t a, int32_t b) {
    return col_ptr[a + 1] - col_ptr[a] < col_ptr[b + 1] - col_ptr[b];
  });
  d.n_vclass = 0;
  {
    int64_t t = 0;
    bool fits = true;
    for (int32_t q = 0; q < n; ++q) {
      const int32_t i = vnode[q], deg = col_ptr[i + 1] - col_ptr[i];
      if (q == 0 || deg != d.vclass_deg[d.n_vclass - 1]) {
        if (d.n_vclass == kMaxVClasses) { fits = false; break; }
        d.vclass_deg[d.n_vclass] = deg;
        d.vclass_first[d.n_vclass] = q;
        d.vclass_toff[d.n_vclass] = t;
        ++d.n_vclass;
      }
      for (int32_t a = col_ptr[i]; a < col_ptr[i + 1]; ++a) {
        vslot[t] = col_slot[a];
        vrow[t++] = slot_row[col_slot[a]];
      }
    }
    if (fits) d.vclass_first[d.n_vclass] = n;
    else d.n_vclass = 0;
  }

  // ---- one device block for every array
  struct Part { const void* src; size_t bytes; size_t off; };
  std::vector<Part> parts = {
      {slice_base.data(), slice_base.size() * 4, 0}, {slot_col.data(), slot_col.size() * 4, 0},
      {col_ptr.data(), col_ptr.size() * 4, 0},       {col_slot.data(), col_slot.size() * 4, 0},
      {row_ptr.data(), row_ptr.size() * 4, 0},       {col_idx.data(), col_idx.size() * 4, 0},
      {edge_slot.data(), edge_slot.size() * 4, 0},   {perm_mat.data(), perm_mat.size(), 0},
      {perm_local.data(), perm_local.size() * 4, 0}, {vnode.data(), vnode.size() * 4, 0},
      {vslot.data(), vslot.size() * 4, 0},           {vrow.data(), vrow.size() * 4, 0},
      {row_at.data(), row_at.size() * 4, 0}};
  size_t total = 0;
  for (auto& p : parts) {
    p.off = total;
    total += (p.bytes + 255) & ~size_t(255);
  }
  mbp_codes* h = new (std::nothrow) mbp_codes{};
  if (!h) return set_error(MBP_ENOMEM, "host allocation failed");
  cudaError_t ce = cudaGetDevice(&h->device);
  if (ce != cudaSuccess) { delete h; return cuda_error(ce, "cudaGetDevice"); }
  ce = cudaMalloc(&h->dev_block, total);
  if (ce != cudaSuccess) {
    delete h;
    cudaGetLastError();
    return set_error(MBP_ENOMEM, "cudaMalloc of %zu bytes for the code failed: %s", total, cudaGetErrorString(ce));
  }
  h->dev_bytes = total;
  char* base = static_cast<char*>(h->dev_block);
  for (auto& p : parts) {
    ce = cudaMemcpy(base + p.off, p.src, p.bytes, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
      cudaFree(h->dev_block);
      delete h;
      return cuda_error(ce, "cudaMemcpy of the code");
    }
  }
  d.slice_base = reinterpret_cast<const int32_t*>(base + parts[0].off);
  d.slot_col = reinterpret_cast<const int32_t*>(base + parts[1].off);
  d.col_ptr = reinterpret_cast<const int32_t*>(base + parts[2].off);
  d.col_slot = reinterpret_cast<const int32_t*>(base + parts[3].off);
  d.row_ptr = reinterpret_cast<const int32_t*>(base + parts[4].off);
  d.col_idx = reinterpret_cast<const int32_t*>(base + parts[5].off);
  d.edge_slot = reinterpret_cast<const int32_t*>(base + parts[6].off);
  d.row_mat = reinterpret_cast<const uint8_t*>(base + parts[7].off);
  d.row_local = reinterpret_cast<const int32_t*>(base + parts[8].off);
  d.vnode = reinterpret_cast<const int32_t*>(base + parts[9].off);
  d.vslot = reinterpret_cast<const int32_t*>(base + parts[10].off);
  // the packed row table holds positions below 2^25; larger codes keep iteration 1 per edge
  d.vrow = m_tot < (int64_t(1) << 25) ? reinterpret_cast<const int32_t*>(base + parts[11].off) : nullptr;
  d.row_at = reinterpret_cast<const int32_t*>(base + parts[12].off);
  h->d = d;
  // The allocation-free decode's scratch lives in this library's device code; looking its address up here,
  // where allocating is allowed, loads that code on this device (lazy module loading would otherwise do so
  // inside the first allocation-free call).
  // A failure here is not the upload's: the allocation-free call repeats the look-up and reports it.
  void* scratch = nullptr;
  if (static_scratch(&scratch) != MBP_OK) {
    cudaGetLastError();
    g_err.clear();
  }
  *out = h;
  return MBP_OK;
}

int mbp_destroy_codes(mbp_codes* codes) {
  g_err.clear();
  if (!codes) return MBP_OK;
  cudaError_t e = cudaDeviceSynchronize();
  multi_forget(codes);  // a later handle may get this address
  cudaError_t f = cudaFree(codes->dev_block);
  delete codes;
  if (e != cudaSuccess) return cuda_error(e, "cudaDeviceSynchronize");
  if (f != cudaSuccess) return cuda_error(f, "cudaFree");
  return MBP_OK;
}

int mbp_codes_info(const mbp_codes* c, int32_t* u, int32_t* n, int32_t* m_total, int64_t* edges,
                   int32_t* max_check_degree) {
  g_err.clear();
  REQUIRE(c, "codes is NULL");
  if (u) *u = c->d.u;
  if (n) *n = c->d.n;
  if (m_total) *m_total = c->d.m_tot;
  if (edges) *edges = c->d.e_tot;
  if (max_check_degree) *max_check_degree = c->d.max_row_deg;
  return MBP_OK;
}

int mbp_syndrome(const mbp_codes* codes, const uint32_t* x_bits, int F, uint32_t* z_bits, mbp_stream_t stream) {
  g_err.clear();
  REQUIRE(codes, "codes is NULL");
  REQUIRE(F >= 0, "F must be >= 0");
  if (F == 0) return MBP_OK;
  REQUIRE_CODES_HERE(codes);
  REQUIRE_DEV(x_bits, "x_bits");
  REQUIRE_DEV(z_bits, "z_bits");
  cudaError_t e = launch_syndrome(codes->d, x_bits, F, z_bits, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? MBP_OK : cuda_error(e, "syndrome kernel");
}

int mbp_bsc_llr(const uint32_t* y_bits, const double* qber, int F, int n, int dtype, void* llr,
                mbp_stream_t stream) {
  g_err.clear();
  REQUIRE(F >= 0 && n > 0, "F must be >= 0 and n > 0");
  REQUIRE(dtype == MBP_MSG_F32 || dtype == MBP_MSG_F64, "unknown dtype %d", dtype);
  if (F == 0) return MBP_OK;
  REQUIRE_DEV(y_bits, "y_bits");
  REQUIRE_DEV(qber, "qber");
  REQUIRE_DEV(llr, "llr");
  cudaError_t e = launch_bsc_llr(y_bits, qber, F, n, dtype, llr, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? MBP_OK : cuda_error(e, "bsc_llr kernel");
}

int mbp_decode_workspace_size(const mbp_codes* codes, int F, const mbp_opts* opts, size_t* bytes) {
  g_err.clear();
  REQUIRE(codes && bytes, "codes and bytes must be non-NULL");
  REQUIRE(F >= 0, "F must be >= 0");
  int rc = validate_opts(opts);
  if (rc) return rc;
  return single_workspace(codes, F, opts, opts->host_io != 0, bytes);
}

static int decode_common(const mbp_codes* codes, int F, const void* llr, const uint32_t* y_bits,
                         const double* qber, const uint32_t* z_bits, int max_iter, const mbp_opts* opts,
                         uint32_t* x_hat_bits, int32_t* iters, uint8_t* success, mbp_stream_t stream) {
  int rc = common_decode_checks(codes, F, max_iter, opts);
  if (rc || F == 0) return rc;
  if (llr) REQUIRE_DEV(llr, "llr");
  if (y_bits) {
    REQUIRE_DEV(y_bits, "y_bits");
    REQUIRE_DEV(qber, "qber");
  }
  REQUIRE_DEV(z_bits, "z_bits");
  REQUIRE_DEV(x_hat_bits, "x_hat_bits");
  REQUIRE_DEV(iters, "iters");
  REQUIRE_DEV(success, "success");
  if (opts->soft_out) REQUIRE_DEV(opts->soft_out, "opts->soft_out");
  if (opts->synd_ok) REQUIRE_DEV(opts->synd_ok, "opts->synd_ok");
  if (graph_schedule(opts)) {
    mbp_group g = one_group(codes, F);
    g.llr = llr;
    g.y_bits = y_bits;
    g.qber = qber;
    g.z_bits = z_bits;
    g.x_hat_bits = x_hat_bits;
    g.iters = iters;
    g.success = success;
    g.synd_ok = opts->synd_ok;
    g.soft_out = opts->soft_out;
    return multi_decode(&g, 1, max_iter, opts, opts->host_io != 0, reinterpret_cast<cudaStream_t>(stream));
  }
  DevState st;
  carve_workspace(codes->d, F, opts->msg_dtype, opts->host_io != 0, opts->workspace, &st);
  DecodeArgs a{};
  a.llr = llr;
  a.y_bits = y_bits;
  a.qber = qber;
  a.z_bits = z_bits;
  a.max_iter = max_iter;
  a.early_exit = opts->early_exit;
  a.accumulate = opts->accumulate;
  a.schedule = opts->schedule;
  a.rule = opts->rule;
  a.update = opts->update;
  a.validate = opts->validate;
  a.l_max = opts->l_max;
  a.x_hat_bits = x_hat_bits;
  a.iters = iters;
  a.success = success;
  a.soft_out = opts->soft_out;
  a.synd_ok = opts->synd_ok;
  return decode(codes->d, st, opts->msg_dtype, a, reinterpret_cast<cudaStream_t>(stream));
}

int mbp_decode_batch(const mbp_codes* codes, int F, const void* llr, const uint32_t* z_bits, int max_iter,
                     const mbp_opts* opts, uint32_t* x_hat_bits, int32_t* iters, uint8_t* success,
                     mbp_stream_t stream) {
  g_err.clear();
  if (F > 0) REQUIRE(llr, "llr is NULL");
  return decode_common(codes, F, llr, nullptr, nullptr, z_bits, max_iter, opts, x_hat_bits, iters, success, stream);
}

int mbp_decode_bsc(const mbp_codes* codes, int F, const uint32_t* y_bits, const double* qber,
                   const uint32_t* z_bits, int max_iter, const mbp_opts* opts, uint32_t* x_hat_bits,
                   int32_t* iters, uint8_t* success, mbp_stream_t stream) {
  g_err.clear();
  if (F > 0) REQUIRE(y_bits && qber, "y_bits and qber must be non-NULL");
  return decode_common(codes, F, nullptr, y_bits, qber, z_bits, max_iter, opts, x_hat_bits, iters, success,
                       stream);
}

}  // extern "C"

// The host-memory decode: inputs copied into the workspace's staging buffers, the decode, the outputs copied
// back; with sync, the call waits for the stream at the end.
static int decode_bsc_host(const mbp_codes* codes, int F, const uint32_t* y_bits, const double* qber,
                           const uint32_t* z_bits, int max_iter, const mbp_opts* opts, uint32_t* x_hat_bits,
                           int32_t* iters, uint8_t* success, mbp_stream_t stream, bool sync) {
  int rc = common_decode_checks(codes, F, max_iter, opts);
  if (rc || F == 0) return rc;
  REQUIRE(opts->host_io == 1, "opts->host_io must be 1 for mbp_decode_bsc_host");
  REQUIRE(y_bits && qber && z_bits && x_hat_bits && iters && success, "host buffers must be non-NULL");
  REQUIRE(opts->soft_out == nullptr || is_device_ptr(opts->soft_out), "opts->soft_out must be a device pointer");
  REQUIRE(opts->synd_ok == nullptr || is_device_ptr(opts->synd_ok), "opts->synd_ok must be a device pointer");
  const DevCode& d = codes->d;
  DevState st;
  if ((rc = single_state(codes, F, opts, true, opts->workspace, &st))) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t wn = (size_t(d.n) + 31) / 32;
  size_t zw = 0;
  for (int l = 0; l < d.u; ++l) zw += (size_t(d.m[l]) + 31) / 32;
  cudaError_t e;
#define CK(call, what) \
  if ((e = (call)) != cudaSuccess) return cuda_error(e, what)
  CK(cudaMemcpyAsync(st.io_y, y_bits, size_t(F) * wn * 4, cudaMemcpyHostToDevice, s), "copy y_bits to device");
  CK(cudaMemcpyAsync(st.io_qber, qber, size_t(F) * 8, cudaMemcpyHostToDevice, s), "copy qber to device");
  CK(cudaMemcpyAsync(st.io_z, z_bits, size_t(F) * zw * 4, cudaMemcpyHostToDevice, s), "copy z_bits to device");
  DecodeArgs a{};
  a.y_bits = st.io_y;
  a.qber = st.io_qber;
  a.z_bits = st.io_z;
  a.max_iter = max_iter;
  a.early_exit = opts->early_exit;
  a.accumulate = opts->accumulate;
  a.schedule = opts->schedule;
  a.rule = opts->rule;
  a.update = opts->update;
  a.validate = opts->validate;
  a.l_max = opts->l_max;
  a.x_hat_bits = st.io_xhat;
  a.iters = st.io_iters;
  a.success = st.io_success;
  a.soft_out = opts->soft_out;
  a.synd_ok = opts->synd_ok;
  if (graph_schedule(opts)) {
    mbp_group g = one_group(codes, F);
    g.y_bits = st.io_y;
    g.qber = st.io_qber;
    g.z_bits = st.io_z;
    g.x_hat_bits = st.io_xhat;
    g.iters = st.io_iters;
    g.success = st.io_success;
    g.synd_ok = opts->synd_ok;
    g.soft_out = opts->soft_out;
    rc = multi_decode(&g, 1, max_iter, opts, true, s);
  } else {
    rc = decode(d, st, opts->msg_dtype, a, s);
  }
  if (rc) return rc;
  CK(cudaMemcpyAsync(x_hat_bits, st.io_xhat, size_t(F) * wn * 4, cudaMemcpyDeviceToHost, s), "copy x_hat to host");
  CK(cudaMemcpyAsync(iters, st.io_iters, size_t(F) * 4, cudaMemcpyDeviceToHost, s), "copy iters to host");
  CK(cudaMemcpyAsync(success, st.io_success, size_t(F), cudaMemcpyDeviceToHost, s), "copy success to host");
  if (sync) CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
#undef CK
  return MBP_OK;
}

extern "C" {

int mbp_decode_bsc_host(const mbp_codes* codes, int F, const uint32_t* y_bits, const double* qber,
                        const uint32_t* z_bits, int max_iter, const mbp_opts* opts, uint32_t* x_hat_bits,
                        int32_t* iters, uint8_t* success, mbp_stream_t stream) {
  g_err.clear();
  return decode_bsc_host(codes, F, y_bits, qber, z_bits, max_iter, opts, x_hat_bits, iters, success, stream, true);
}

int mbp_decode_bsc_host_async(const mbp_codes* codes, int F, const uint32_t* y_bits, const double* qber,
                              const uint32_t* z_bits, int max_iter, const mbp_opts* opts, uint32_t* x_hat_bits,
                              int32_t* iters, uint8_t* success, mbp_stream_t stream) {
  g_err.clear();
  return decode_bsc_host(codes, F, y_bits, qber, z_bits, max_iter, opts, x_hat_bits, iters, success, stream, false);
}

int mbp_decode_bsc_static(const mbp_codes* codes, int F, const uint32_t* y_bits, const double* qber,
                          const uint32_t* z_bits, int max_iter, const mbp_opts* opts, uint32_t* x_hat_bits,
                          int32_t* iters, uint8_t* success, mbp_stream_t stream) {
  g_err.clear();
  REQUIRE(codes, "codes is NULL");
  REQUIRE(F >= 0, "F must be >= 0");
  REQUIRE(max_iter >= 0 && max_iter <= 1000000, "max_iter must be in [0, 1e6]");
  if (F == 0) return MBP_OK;
  int rc = validate_opts(opts);
  if (rc) return rc;
  REQUIRE_CODES_HERE(codes);
  REQUIRE(opts->host_io == 0, "opts->host_io must be 0 for mbp_decode_bsc_static");
  if (opts->schedule == MBP_SCHED_GRAPH)  // instantiating a CUDA graph may allocate; AUTO runs the streaming one
    return set_error(MBP_EUNSUPPORTED, "mbp_decode_bsc_static runs the streaming or resident schedule only");
  const size_t need = workspace_bytes(codes->d, F, opts->msg_dtype, false);
  REQUIRE(need <= MBP_STATIC_SCRATCH_BYTES,
          "F = %d needs %zu bytes of decoder state, more than the %u bytes of static scratch", F, need,
          MBP_STATIC_SCRATCH_BYTES);
  REQUIRE(y_bits && qber, "y_bits and qber must be non-NULL");
  REQUIRE_DEV(y_bits, "y_bits");
  REQUIRE_DEV(qber, "qber");
  REQUIRE_DEV(z_bits, "z_bits");
  REQUIRE_DEV(x_hat_bits, "x_hat_bits");
  REQUIRE_DEV(iters, "iters");
  REQUIRE_DEV(success, "success");
  if (opts->soft_out) REQUIRE_DEV(opts->soft_out, "opts->soft_out");
  if (opts->synd_ok) REQUIRE_DEV(opts->synd_ok, "opts->synd_ok");
  void* scratch = nullptr;
  rc = static_scratch(&scratch);
  if (rc) return rc;
  DevState st;
  carve_workspace(codes->d, F, opts->msg_dtype, false, scratch, &st);
  DecodeArgs a{};
  a.y_bits = y_bits;
  a.qber = qber;
  a.z_bits = z_bits;
  a.max_iter = max_iter;
  a.early_exit = opts->early_exit;
  a.accumulate = opts->accumulate;
  a.schedule = opts->schedule;
  a.rule = opts->rule;
  a.update = opts->update;
  a.validate = 0;
  a.l_max = opts->l_max;
  a.x_hat_bits = x_hat_bits;
  a.iters = iters;
  a.success = success;
  a.soft_out = opts->soft_out;
  a.synd_ok = opts->synd_ok;
  return decode(codes->d, st, opts->msg_dtype, a, reinterpret_cast<cudaStream_t>(stream));
}

int mbp_export_c2v(const mbp_codes* codes, int F, const mbp_opts* opts, int frame, void* c2v_out,
                   mbp_stream_t stream) {
  g_err.clear();
  REQUIRE(codes, "codes is NULL");
  REQUIRE(F > 0 && frame >= 0 && frame < F, "frame %d outside [0, F = %d)", frame, F);
  REQUIRE_CODES_HERE(codes);
  int rc = validate_opts(opts);
  if (rc) return rc;
  rc = check_workspace(codes, F, opts);
  if (rc) return rc;
  REQUIRE_DEV(c2v_out, "c2v_out");
  DevState st;
  if ((rc = single_state(codes, F, opts, opts->host_io != 0, opts->workspace, &st))) return rc;
  cudaError_t e = launch_export_c2v(codes->d, st, opts->msg_dtype, frame, c2v_out,
                                    reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? MBP_OK : cuda_error(e, "export kernel");
}

static int check_groups(const mbp_group* g, int G, const mbp_opts* o, bool need_workspace) {
  REQUIRE(G >= 0 && G <= kMaxGroups, "G = %d outside [0, %d]", G, kMaxGroups);
  REQUIRE(G == 0 || g, "groups is NULL");
  int rc = validate_opts(o);
  if (rc) return rc;
  if ((rc = multi_check_opts(o))) return rc;
  int64_t tiles = 0;
  for (int i = 0; i < G; ++i) {
    REQUIRE(g[i].codes, "group %d: codes is NULL", i);
    REQUIRE(g[i].F >= 0, "group %d: F must be >= 0", i);
    if (need_workspace && g[i].F > 0) REQUIRE_CODES_HERE(g[i].codes);
    tiles += (g[i].F + kLanes - 1) / kLanes;
  }
  if (tiles > 65535) return set_error(MBP_EUNSUPPORTED, "a batch may hold at most %d frames", 65535 * kLanes);
  if (!need_workspace) return MBP_OK;
  for (int i = 0; i < G; ++i) {
    if (g[i].F == 0) continue;
    if (g[i].llr) {
      REQUIRE(is_device_ptr(g[i].llr), "group %d: llr must be a device pointer", i);
    } else {
      REQUIRE(is_device_ptr(g[i].y_bits) && is_device_ptr(g[i].qber),
              "group %d: y_bits and qber must be device pointers when llr is NULL", i);
    }
    REQUIRE(is_device_ptr(g[i].z_bits), "group %d: z_bits must be a device pointer", i);
    REQUIRE(is_device_ptr(g[i].x_hat_bits), "group %d: x_hat_bits must be a device pointer", i);
    REQUIRE(is_device_ptr(g[i].iters), "group %d: iters must be a device pointer", i);
    REQUIRE(is_device_ptr(g[i].success), "group %d: success must be a device pointer", i);
    REQUIRE(!g[i].synd_ok || is_device_ptr(g[i].synd_ok), "group %d: synd_ok must be a device pointer", i);
    REQUIRE(!g[i].soft_out || is_device_ptr(g[i].soft_out), "group %d: soft_out must be a device pointer", i);
  }
  size_t need = 0;
  if ((rc = multi_workspace(g, G, o, false, &need))) return rc;
  REQUIRE(o->workspace, "opts->workspace is NULL (size it with mbp_multi_workspace_size)");
  REQUIRE((reinterpret_cast<uintptr_t>(o->workspace) & 255) == 0, "workspace must be 256-byte aligned");
  REQUIRE(o->workspace_bytes >= need, "workspace too small: %zu bytes given, %zu needed", o->workspace_bytes, need);
  REQUIRE_DEV(o->workspace, "workspace");
  return MBP_OK;
}

int mbp_multi_workspace_size(const mbp_group* groups, int G, const mbp_opts* opts, size_t* bytes) {
  g_err.clear();
  REQUIRE(bytes, "bytes is NULL");
  int rc = check_groups(groups, G, opts, false);
  if (rc) return rc;
  return multi_workspace(groups, G, opts, false, bytes);
}

int mbp_decode_multi(const mbp_group* groups, int G, int max_iter, const mbp_opts* opts, mbp_stream_t stream) {
  g_err.clear();
  REQUIRE(max_iter >= 0 && max_iter <= 1000000, "max_iter must be in [0, 1e6]");
  int rc = check_groups(groups, G, opts, true);
  if (rc) return rc;
  return multi_decode(groups, G, max_iter, opts, false, reinterpret_cast<cudaStream_t>(stream));
}

int mbp_autotune_multi(const mbp_group* groups, int G, int max_iter, const mbp_opts* opts, mbp_tuning* best,
                       mbp_stream_t stream) {
  g_err.clear();
  REQUIRE(max_iter >= 0 && max_iter <= 1000000, "max_iter must be in [0, 1e6]");
  int rc = check_groups(groups, G, opts, true);
  if (rc) return rc;
  return multi_autotune(groups, G, max_iter, opts, best, reinterpret_cast<cudaStream_t>(stream));
}

int mbp_multi_set_tuning(const mbp_group* groups, int G, const mbp_opts* opts, const mbp_tuning* tuning) {
  g_err.clear();
  REQUIRE(tuning, "tuning is NULL");
  int rc = check_groups(groups, G, opts, false);
  if (rc) return rc;
  auto ok = [](int w) { return w == 2 || w == 4 || w == 8; };
  REQUIRE(ok(tuning->cn_warps) && ok(tuning->vn_warps) && ok(tuning->syn_warps) &&
              (tuning->cn_waves == 1 || tuning->cn_waves == 2),
          "tuning: warps per block must be 2, 4 or 8 and cn_waves 1 or 2");
  return multi_set_tuning(groups, G, opts, tuning);
}

int mbp_release_cached(void) {
  g_err.clear();
  multi_release();
  return MBP_OK;
}

static int check_nbp(const mbp_codes* codes, int F, int T, double l_max, const void* ws, size_t ws_bytes) {
  REQUIRE(codes, "codes is NULL");
  REQUIRE(F >= 0 && T >= 1 && T <= 1000, "F must be >= 0 and T in [1, 1000]");
  REQUIRE(std::isfinite(l_max) && l_max > 0, "l_max must be finite and > 0");
  if (codes->d.max_row_deg > 32)
    return set_error(MBP_EUNSUPPORTED, "the unrolled decoder supports checks of at most 32 edges");
  if (F == 0) return MBP_OK;
  REQUIRE_CODES_HERE(codes);
  if ((F + kLanes - 1) / kLanes > 65535) return set_error(MBP_EUNSUPPORTED, "F = %d is too large", F);
  const size_t need = nbp_workspace_bytes(codes->d, F, T);
  REQUIRE(ws, "workspace is NULL (size it with mbp_nbp_workspace_size)");
  REQUIRE((reinterpret_cast<uintptr_t>(ws) & 255) == 0, "workspace must be 256-byte aligned");
  REQUIRE(ws_bytes >= need, "workspace too small: %zu bytes given, %zu needed", ws_bytes, need);
  REQUIRE_DEV(ws, "workspace");
  return MBP_OK;
}

int mbp_nbp_workspace_size(const mbp_codes* codes, int F, int T, size_t* bytes) {
  g_err.clear();
  REQUIRE(codes && bytes, "codes and bytes must be non-NULL");
  REQUIRE(F >= 0 && T >= 1 && T <= 1000, "F must be >= 0 and T in [1, 1000]");
  *bytes = nbp_workspace_bytes(codes->d, F, T);
  return MBP_OK;
}

int mbp_nbp_forward(const mbp_codes* codes, int F, int T, const float* llr, const uint32_t* z_bits,
                    const float* alpha, const float* beta, double l_max, void* workspace, size_t workspace_bytes,
                    float* lv_out, mbp_stream_t stream) {
  g_err.clear();
  int rc = check_nbp(codes, F, T, l_max, workspace, workspace_bytes);
  if (rc || F == 0) return rc;
  REQUIRE_DEV(llr, "llr");
  REQUIRE_DEV(z_bits, "z_bits");
  REQUIRE_DEV(alpha, "alpha");
  REQUIRE_DEV(beta, "beta");
  if (lv_out) REQUIRE_DEV(lv_out, "lv_out");
  DevState st;
  NbpState ns;
  nbp_carve(codes->d, F, T, workspace, &st, &ns);
  return nbp_forward(codes->d, st, ns, llr, z_bits, alpha, beta, l_max, lv_out,
                     reinterpret_cast<cudaStream_t>(stream));
}

int mbp_nbp_backward(const mbp_codes* codes, int F, int T, const float* alpha, const float* beta, double l_max,
                     const float* grad_lv, void* workspace, size_t workspace_bytes, float* grad_alpha,
                     float* grad_beta, float* grad_llr, mbp_stream_t stream) {
  g_err.clear();
  int rc = check_nbp(codes, F, T, l_max, workspace, workspace_bytes);
  if (rc) return rc;
  REQUIRE_DEV(grad_alpha, "grad_alpha");
  REQUIRE_DEV(grad_beta, "grad_beta");
  if (F == 0) {
    const size_t b = sizeof(float) * size_t(T) * codes->d.u;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(grad_alpha, 0, b, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(grad_beta, 0, b, s);
    return e == cudaSuccess ? MBP_OK : cuda_error(e, "clear gradients");
  }
  REQUIRE_DEV(alpha, "alpha");
  REQUIRE_DEV(beta, "beta");
  REQUIRE_DEV(grad_lv, "grad_lv");
  if (grad_llr) REQUIRE_DEV(grad_llr, "grad_llr");
  DevState st;
  NbpState ns;
  nbp_carve(codes->d, F, T, workspace, &st, &ns);
  return nbp_backward(codes->d, ns, alpha, beta, l_max, grad_lv, grad_alpha, grad_beta, grad_llr,
                      reinterpret_cast<cudaStream_t>(stream));
}

int mbp_profile_enable(int on) {
  g_err.clear();
  prof_enable(on != 0);
  return MBP_OK;
}

int mbp_profile_get(int family, int64_t* launches, double* milliseconds) {
  g_err.clear();
  return prof_get(family, launches, milliseconds);
}

}  // extern "C"
