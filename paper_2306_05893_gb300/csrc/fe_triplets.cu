// Generic triplet ingestion (Section 4.2): a caller's (row, col, value)
// stream in its own filling order, the filling-order test of Algorithm
// "add", the pattern by two counting-sort transposes through the
// uncompressed structure (Table "build pattern"), and the per-step merge of
// the values through the map C on the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/fe_hotpath.h"

struct fe_trip {
  int64_t n = 0;
  int device = 0;
  int64_t ntrip = -1;                    // -1: no stream seen yet
  std::vector<int32_t> rows, cols;       // host copy of the last (row, col) stream
  std::vector<int32_t> rowptr, colind, C;
  std::vector<int64_t> slot_ptr;         // [nnz + 1] into slot_src
  std::vector<int32_t> slot_src;         // triplet ids of every slot, ascending
  int64_t nnz = 0;
  // device copies (capacities in elements)
  int32_t *d_rows = nullptr, *d_cols = nullptr, *d_rowptr = nullptr, *d_colind = nullptr, *d_slot_src = nullptr;
  int64_t *d_slot_ptr = nullptr;
  double *d_vals = nullptr, *d_A = nullptr;
  int *d_flag = nullptr, *h_flag = nullptr;
  int64_t cap_trip = 0, cap_nnz = 0;
  std::string err;
};

namespace {

int fail(fe_trip *t, int code, const std::string &m) {
  t->err = m;
  return code;
}

#define TRIP_CUDA(call)                                                              \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      cudaGetLastError();                                                            \
      return fail(t, FE_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    }                                                                                \
  } while (0)

// 1 in *flag when the streams differ anywhere
__global__ void trip_compare_kernel(int64_t m, const int32_t *__restrict__ r, const int32_t *__restrict__ c,
                                    const int32_t *__restrict__ pr, const int32_t *__restrict__ pc, int *flag) {
  bool diff = false;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x)
    diff |= (r[i] != pr[i]) | (c[i] != pc[i]);
  if (__syncthreads_or(diff) && threadIdx.x == 0) atomicOr(flag, 1);
}

// A[s] = sum of vals over slot s's triplets, in ascending stream order
__global__ void trip_merge_kernel(int64_t nnz, const int64_t *__restrict__ slot_ptr,
                                  const int32_t *__restrict__ slot_src, const double *__restrict__ vals,
                                  double *__restrict__ A) {
  for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < nnz; s += int64_t(gridDim.x) * blockDim.x) {
    double acc = 0.0;
    const int64_t k1 = slot_ptr[s + 1];
    for (int64_t k = slot_ptr[s]; k < k1; ++k) acc += vals[slot_src[k]];
    A[s] = acc;
  }
}

unsigned grid_of(int64_t m) { return unsigned(std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 152 * 16))); }

// Full assembly of the pattern: X^T then (X^T)^T in the uncompressed
// structure (counting sorts by column, then by row, each stable in the
// stream order), then the merge of equal positions into CSR, the slot lists
// and C.
int build_pattern(fe_trip *t) {
  const int64_t n = t->n, m = t->ntrip;
  for (int64_t i = 0; i < m; ++i)
    if (t->rows[i] < 0 || t->rows[i] >= n || t->cols[i] < 0 || t->cols[i] >= n)
      return fail(t, FE_ERR_ARG, "triplet " + std::to_string(i) + " lies outside the n x n matrix");
  std::vector<int64_t> colptr(n + 1, 0);
  for (int64_t i = 0; i < m; ++i) colptr[t->cols[i] + 1]++;
  for (int64_t j = 0; j < n; ++j) colptr[j + 1] += colptr[j];
  std::vector<int32_t> xt_row(m), xt_id(m);
  {
    std::vector<int64_t> next(colptr.begin(), colptr.end() - 1);
    for (int64_t i = 0; i < m; ++i) {
      const int64_t p = next[t->cols[i]]++;
      xt_row[p] = t->rows[i];
      xt_id[p] = int32_t(i);
    }
  }
  std::vector<int64_t> rp(n + 1, 0);
  for (int64_t p = 0; p < m; ++p) rp[xt_row[p] + 1]++;
  for (int64_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
  std::vector<int32_t> x_col(m);
  t->slot_src.assign(m, 0);
  {
    std::vector<int64_t> next(rp.begin(), rp.end() - 1);
    for (int64_t j = 0; j < n; ++j)
      for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
        const int64_t q = next[xt_row[p]]++;
        x_col[q] = int32_t(j);
        t->slot_src[q] = xt_id[p];
      }
  }
  t->rowptr.assign(n + 1, 0);
  t->colind.clear();
  t->slot_ptr.clear();
  t->C.assign(m, 0);
  for (int64_t i = 0; i < n; ++i) {
    t->rowptr[i] = int32_t(t->colind.size());
    int32_t last = -1;
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
      if (x_col[q] != last) {
        last = x_col[q];
        t->slot_ptr.push_back(q);
        t->colind.push_back(last);
      }
      t->C[t->slot_src[q]] = int32_t(t->colind.size() - 1);
    }
  }
  t->nnz = int64_t(t->colind.size());
  t->rowptr[n] = int32_t(t->nnz);
  t->slot_ptr.push_back(m);
  return FE_OK;
}

template <typename T>
int grow(fe_trip *t, T **p, int64_t need, int64_t have) {
  if (need <= have && *p) return FE_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  TRIP_CUDA(cudaMalloc(reinterpret_cast<void **>(p), size_t(std::max<int64_t>(need, 1)) * sizeof(T)));
  return FE_OK;
}

int upload_pattern(fe_trip *t, cudaStream_t s) {
  const int64_t m = std::max<int64_t>(t->ntrip, 1), z = std::max<int64_t>(t->nnz, 1);
  int st;
  if ((st = grow(t, &t->d_rows, m, t->cap_trip)) || (st = grow(t, &t->d_cols, m, t->cap_trip)) ||
      (st = grow(t, &t->d_slot_src, m, t->cap_trip)) || (st = grow(t, &t->d_vals, m, t->cap_trip)))
    return st;
  t->cap_trip = std::max(t->cap_trip, m);
  if ((st = grow(t, &t->d_colind, z, t->cap_nnz)) || (st = grow(t, &t->d_slot_ptr, z + 1, t->cap_nnz + 1)) ||
      (st = grow(t, &t->d_A, z, t->cap_nnz)))
    return st;
  t->cap_nnz = std::max(t->cap_nnz, z);
  if (t->ntrip > 0) {
    TRIP_CUDA(cudaMemcpyAsync(t->d_rows, t->rows.data(), t->ntrip * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    TRIP_CUDA(cudaMemcpyAsync(t->d_cols, t->cols.data(), t->ntrip * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    TRIP_CUDA(cudaMemcpyAsync(t->d_slot_src, t->slot_src.data(), t->ntrip * sizeof(int32_t),
                              cudaMemcpyHostToDevice, s));
  }
  TRIP_CUDA(cudaMemcpyAsync(t->d_rowptr, t->rowptr.data(), (t->n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  if (t->nnz > 0)
    TRIP_CUDA(cudaMemcpyAsync(t->d_colind, t->colind.data(), t->nnz * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  TRIP_CUDA(cudaMemcpyAsync(t->d_slot_ptr, t->slot_ptr.data(), (t->nnz + 1) * sizeof(int64_t),
                            cudaMemcpyHostToDevice, s));
  // the host vectors are read by the copies above: finish them before any change
  TRIP_CUDA(cudaStreamSynchronize(s));
  return FE_OK;
}

}  // namespace

extern "C" {

int fe_trip_create(int64_t n, fe_trip **out) {
  if (!out) return FE_ERR_ARG;
  *out = nullptr;
  if (n < 1 || n >= (int64_t(1) << 31)) return FE_ERR_ARG;
  fe_trip *t = new (std::nothrow) fe_trip();
  if (!t) return FE_ERR_OOM;
  t->n = n;
  if (cudaGetDevice(&t->device) != cudaSuccess || cudaMalloc(&t->d_rowptr, (n + 1) * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&t->d_flag, sizeof(int)) != cudaSuccess || cudaMallocHost(&t->h_flag, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    fe_trip_destroy(t);
    return FE_ERR_CUDA;
  }
  *out = t;
  return FE_OK;
}

int fe_trip_assemble(fe_trip *t, int64_t ntrip, const int32_t *rows, const int32_t *cols, const double *vals,
                     int32_t device_ptrs, void *stream, int32_t *rebuilt) {
  if (!t) return FE_ERR_ARG;
  if (ntrip < 0 || ntrip >= (int64_t(1) << 31) || (ntrip > 0 && (!rows || !cols || !vals)))
    return fail(t, FE_ERR_ARG, "bad triplet arrays");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // filling-order test (Algorithm "add"): same length and same (row, col) at every position
  bool keep = (t->ntrip == ntrip);
  if (keep && ntrip > 0) {
    if (device_ptrs) {
      TRIP_CUDA(cudaMemsetAsync(t->d_flag, 0, sizeof(int), s));
      trip_compare_kernel<<<grid_of(ntrip), 256, 0, s>>>(ntrip, rows, cols, t->d_rows, t->d_cols, t->d_flag);
      TRIP_CUDA(cudaGetLastError());
      TRIP_CUDA(cudaMemcpyAsync(t->h_flag, t->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
      TRIP_CUDA(cudaStreamSynchronize(s));
      keep = (*t->h_flag == 0);
    } else {
      keep = std::memcmp(rows, t->rows.data(), ntrip * sizeof(int32_t)) == 0 &&
             std::memcmp(cols, t->cols.data(), ntrip * sizeof(int32_t)) == 0;
    }
  }
  if (!keep) {  // full assembly of the pattern
    try {
      t->rows.resize(ntrip);
      t->cols.resize(ntrip);
    } catch (const std::bad_alloc &) {
      return fail(t, FE_ERR_OOM, "host allocation failed");
    }
    if (ntrip > 0) {
      if (device_ptrs) {
        TRIP_CUDA(cudaMemcpyAsync(t->rows.data(), rows, ntrip * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        TRIP_CUDA(cudaMemcpyAsync(t->cols.data(), cols, ntrip * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        TRIP_CUDA(cudaStreamSynchronize(s));
      } else {
        std::memcpy(t->rows.data(), rows, ntrip * sizeof(int32_t));
        std::memcpy(t->cols.data(), cols, ntrip * sizeof(int32_t));
      }
    }
    t->ntrip = ntrip;
    int st;
    try {
      st = build_pattern(t);
    } catch (const std::bad_alloc &) {
      st = fail(t, FE_ERR_OOM, "host allocation failed in the pattern build");
    }
    if (st) {
      t->ntrip = -1;  // nothing valid to keep
      return st;
    }
    if ((st = upload_pattern(t, s))) {
      t->ntrip = -1;
      return st;
    }
  }
  if (rebuilt) *rebuilt = keep ? 0 : 1;
  if (ntrip == 0 || t->nnz == 0) return FE_OK;
  const double *dv = vals;
  if (!device_ptrs) {
    TRIP_CUDA(cudaMemcpyAsync(t->d_vals, vals, ntrip * sizeof(double), cudaMemcpyHostToDevice, s));
    dv = t->d_vals;
  }
  trip_merge_kernel<<<grid_of(t->nnz), 256, 0, s>>>(t->nnz, t->d_slot_ptr, t->d_slot_src, dv, t->d_A);
  TRIP_CUDA(cudaGetLastError());
  return FE_OK;
}

int fe_trip_pattern(fe_trip *t, int64_t *nnz, const int32_t **rowptr, const int32_t **colind,
                    const int32_t **scatter) {
  if (!t) return FE_ERR_ARG;
  if (t->ntrip < 0) return fail(t, FE_ERR_STATE, "no triplet stream assembled yet");
  if (nnz) *nnz = t->nnz;
  if (rowptr) *rowptr = t->rowptr.data();
  if (colind) *colind = t->colind.data();
  if (scatter) *scatter = t->C.data();
  return FE_OK;
}

int fe_trip_values(fe_trip *t, double *out, int32_t device_ptrs, void *stream) {
  if (!t || !out) return FE_ERR_ARG;
  if (t->ntrip < 0) return fail(t, FE_ERR_STATE, "no triplet stream assembled yet");
  if (t->nnz == 0) return FE_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  TRIP_CUDA(cudaMemcpyAsync(out, t->d_A, t->nnz * sizeof(double),
                            device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (!device_ptrs) TRIP_CUDA(cudaStreamSynchronize(s));
  return FE_OK;
}

int fe_trip_device_csr(fe_trip *t, const int32_t **rowptr, const int32_t **colind, const double **vals) {
  if (!t) return FE_ERR_ARG;
  if (t->ntrip < 0) return fail(t, FE_ERR_STATE, "no triplet stream assembled yet");
  if (rowptr) *rowptr = t->d_rowptr;
  if (colind) *colind = t->d_colind;
  if (vals) *vals = t->d_A;
  return FE_OK;
}

const char *fe_trip_last_error(const fe_trip *t) { return t ? t->err.c_str() : "null handle"; }

void fe_trip_destroy(fe_trip *t) {
  if (!t) return;
  for (void *p : {static_cast<void *>(t->d_rows), static_cast<void *>(t->d_cols), static_cast<void *>(t->d_rowptr),
                  static_cast<void *>(t->d_colind), static_cast<void *>(t->d_slot_src),
                  static_cast<void *>(t->d_slot_ptr), static_cast<void *>(t->d_vals), static_cast<void *>(t->d_A),
                  static_cast<void *>(t->d_flag)})
    if (p) cudaFree(p);
  if (t->h_flag) cudaFreeHost(t->h_flag);
  cudaGetLastError();
  delete t;
}

}  // extern "C"
