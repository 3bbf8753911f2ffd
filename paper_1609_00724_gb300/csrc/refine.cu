// Hilbert-curve refinement and the Hilbert -> rectilinear converter
// (Sec. "Adaptive refinements" of arXiv:1609.00724) for sm_103a.
//
// Samples live as structure-of-arrays sorted by Hilbert key (key, q, length,
// faces, status). One refinement iteration:
//   (A) flag every pair adjacent along the curve with key gap > 1 and
//       |L_i - L_i+1| > tau; the new sample is the in-region cell nearest the
//       mean key (the region is the effective lattice; skipping whole
//       out-of-region blocks of the curve when it leaves a clipped box);
//   (B) shifted-curve pass: keys of the lattice shifted by S = 2^(p-1) +- the
//       half coarse spacing (alternating) on a curve of order p+1, sorted, the
//       same flag rule, new cells mapped back by -S;
// after each pass the new samples are traced and merged (radix sort by key).
// The host loop reads one count per pass.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cstring>
#include <utility>
#include <vector>

#include "hilbert_dev.cuh"
#include "qsl_internal.cuh"

namespace qsl {
int run_lines(const qsl_field* f, const SeedSource& src, int64_t S, const qsl_opts* o, const LineOutputs& out,
              cudaStream_t stream);
const DeviceStats* last_run_stats_dev();
}

namespace qsl {
namespace {

const uint64_t NONE = ~0ull;

__global__ void encode_kernel(const uint32_t* __restrict__ c, int64_t n, int nd, int bits, uint64_t* keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t cc[3] = {c[nd * i], c[nd * i + 1], nd == 3 ? c[nd * i + 2] : 0u};
    keys[i] = hilbert_key_dev(cc, nd, bits);
  }
}

__global__ void decode_kernel(const uint64_t* __restrict__ keys, int64_t n, int nd, int bits, uint32_t* c) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t cc[3];
    hilbert_coords_dev(keys[i], nd, bits, cc);
    for (int a = 0; a < nd; ++a) c[nd * i + a] = cc[a];
  }
}

struct Region {
  uint64_t lo[3], hi[3];  // lo <= c < hi per axis
};

__device__ __forceinline__ bool in_region(const uint32_t* c, int nd, const Region& r) {
  for (int a = 0; a < nd; ++a)
    if (c[a] < r.lo[a] || c[a] >= r.hi[a]) return false;
  return true;
}

// In-region cell nearest to key m strictly between k_lo and k_hi along the
// curve (lower one on ties); skips whole aligned out-of-region blocks.
__device__ bool nearest_in_region(uint64_t m, uint64_t k_lo, uint64_t k_hi, int nd, int bits, const Region& r,
                                  uint64_t* out) {
  uint64_t found[2];
  bool have[2] = {false, false};
  for (int d = 0; d < 2; ++d) {
    uint64_t k = m;
    for (int guard = 0; guard < 4096; ++guard) {
      if (k <= k_lo || k >= k_hi) break;
      uint32_t c[3] = {0, 0, 0};
      hilbert_coords_dev(k, nd, bits, c);
      if (in_region(c, nd, r)) {
        found[d] = k;
        have[d] = true;
        break;
      }
      int lev = 0;
      while (lev < bits) {
        int l = lev + 1;
        bool outside = false;
        for (int a = 0; a < nd; ++a) {
          uint64_t b0 = ((uint64_t)c[a] >> l) << l;
          uint64_t b1 = b0 + (1ull << l);
          if (b1 <= r.lo[a] || b0 >= r.hi[a]) outside = true;
        }
        if (!outside) break;
        lev = l;
      }
      uint64_t blk = 1ull << (nd * lev);
      uint64_t start = (k / blk) * blk;
      if (d == 0) {
        if (start == 0) break;
        k = start - 1;
      } else {
        k = start + blk;
      }
    }
  }
  if (have[0] && have[1]) {
    *out = (m - found[0] <= found[1] - m) ? found[0] : found[1];
    return true;
  }
  if (have[0]) {
    *out = found[0];
    return true;
  }
  if (have[1]) {
    *out = found[1];
    return true;
  }
  return false;
}

// Coarse pass keys: cell (i*R + R/2, ...) of the effective lattice.
__global__ void coarse_keys_kernel(int64_t n, int nd, int bits, int R, int nc0, int nc1, uint64_t* keys) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = g % nc0, rem = g / nc0;
    int64_t j = rem % nc1, k = rem / nc1;
    uint32_t c[3] = {(uint32_t)(i * R + R / 2), (uint32_t)(j * R + R / 2), (uint32_t)(k * R + R / 2)};
    keys[g] = hilbert_key_dev(c, nd, bits);
  }
}

// Proposal: the effective cells of the flagged coarse cells at stride `st`
// (offset st / 2) that are not already samples (binary search in the sorted
// keys). One thread per (flagged cell, sub-cell).
__global__ void proposal_keys_kernel(const int64_t* __restrict__ cells, const int64_t* ncells_dev, int nd, int bits,
                                     int R, int st, int nc0, int nc1, const uint64_t* __restrict__ have,
                                     int64_t n_have, uint64_t* keys, int64_t* count) {
  int64_t ncells = *ncells_dev;
  const int Rs = R / st;
  int64_t per = 1;
  for (int a = 0; a < nd; ++a) per *= Rs;
  int64_t total = ncells * per;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t cell = cells[t / per], sub = t % per;
    int64_t i = cell % nc0, rem = cell / nc0;
    int64_t j = rem % nc1, k = rem / nc1;
    int64_t s0 = (sub % Rs) * st + st / 2, s1 = ((sub / Rs) % Rs) * st + st / 2,
            s2 = nd == 3 ? (sub / (Rs * Rs)) * st + st / 2 : 0;
    uint32_t c[3] = {(uint32_t)(i * R + s0), (uint32_t)(j * R + s1), (uint32_t)(k * R + s2)};
    uint64_t key = hilbert_key_dev(c, nd, bits);
    int64_t lo = 0, hi = n_have;  // already a sample?
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (have[mid] < key) lo = mid + 1; else hi = mid;
    }
    if (lo < n_have && have[lo] == key) continue;
    unsigned long long pos = atomicAdd((unsigned long long*)count, 1ull);
    keys[pos] = key;
  }
}

__global__ void mask_cells_kernel(const uint8_t* __restrict__ mask, int64_t n, int64_t* cells, int64_t* count) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    if (mask[g]) {
      unsigned long long pos = atomicAdd((unsigned long long*)count, 1ull);
      cells[pos] = g;
    }
  }
}

// Pass A flags: candidate key per pair, NONE when not refined.
// Refinement criterion of a pair of samples adjacent along a curve, on the
// criterion value v of each (L for the FLL jump, Q for the Q threshold).
struct Criterion {
  int kind;  // QSL_REFINE_FLL_JUMP or QSL_REFINE_Q_THRESHOLD
  double tau, q_threshold;
};

__device__ __forceinline__ bool pair_flagged(const Criterion& cr, float va, float vb) {
  if (cr.kind == QSL_REFINE_Q_THRESHOLD)
    return (isfinite(va) && (double)va > cr.q_threshold) || (isfinite(vb) && (double)vb > cr.q_threshold);
  return fabs((double)vb - (double)va) > cr.tau;
}

__global__ void flag_pairs_kernel(const uint64_t* __restrict__ keys, const float* __restrict__ V, int64_t n,
                                  Criterion cr, int nd, int bits, Region reg, uint64_t* cand, int64_t* flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i + 1 < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t a = keys[i], b = keys[i + 1];
    uint64_t out = NONE;
    if (b - a > 1 && pair_flagged(cr, V[i], V[i + 1])) {
      uint64_t got;
      if (nearest_in_region(a + (b - a) / 2, a, b, nd, bits, reg, &got)) out = got;
    }
    cand[i] = out;
    flags[i] = out != NONE;
  }
}

// Shifted keys of all samples (curve of order p+1).
__global__ void shift_keys_kernel(const uint64_t* __restrict__ keys, int64_t n, int nd, int bits, uint32_t S,
                                  uint64_t* skeys, int64_t* perm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[3] = {0, 0, 0};
    hilbert_coords_dev(keys[i], nd, bits, c);
    for (int a = 0; a < nd; ++a) c[a] += S;
    skeys[i] = hilbert_key_dev(c, nd, bits + 1);
    perm[i] = i;
  }
}

// Pass B flags along the shifted curve; candidates are keys on the original curve.
__global__ void flag_shifted_kernel(const uint64_t* __restrict__ skeys, const float* __restrict__ sV, int64_t n,
                                    Criterion cr, int nd, int bits, uint32_t S, Region sreg, uint64_t* cand,
                                    int64_t* flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i + 1 < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t a = skeys[i], b = skeys[i + 1];
    uint64_t out = NONE;
    if (b - a > 1 && pair_flagged(cr, sV[i], sV[i + 1])) {
      uint64_t got;
      if (nearest_in_region(a + (b - a) / 2, a, b, nd, bits + 1, sreg, &got)) {
        uint32_t c[3] = {0, 0, 0};
        hilbert_coords_dev(got, nd, bits + 1, c);
        for (int a2 = 0; a2 < nd; ++a2) c[a2] -= S;
        out = hilbert_key_dev(c, nd, bits);
      }
    }
    cand[i] = out;
    flags[i] = out != NONE;
  }
}

// Shifted keys of samples given by key, with their criterion values looked up
// in the sorted set (key[0..n), V), perm = identity.
__global__ void shift_lookup_kernel(const uint64_t* __restrict__ qkeys, int64_t m, int nd, int bits, uint32_t S,
                                    const uint64_t* __restrict__ key, int64_t n, const float* __restrict__ V,
                                    uint64_t* skeys, float* vals, int64_t* perm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = qkeys[i];
    uint32_t c[3] = {0, 0, 0};
    hilbert_coords_dev(k, nd, bits, c);
    for (int a = 0; a < nd; ++a) c[a] += S;
    skeys[i] = hilbert_key_dev(c, nd, bits + 1);
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (key[mid] < k) lo = mid + 1;
      else hi = mid;
    }
    vals[i] = (lo < n && key[lo] == k) ? V[lo] : __int_as_float(0x7fc00000);
    perm[i] = i;
  }
}

// Stream compaction of candidates != NONE: scatter by the exclusive scan of their flags.
__global__ void cand_scatter_kernel(const uint64_t* __restrict__ cand, const int64_t* __restrict__ pos, int64_t n,
                                    int64_t limit, uint64_t* out, int64_t* count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (cand[i] != NONE && pos[i] < limit) out[pos[i]] = cand[i];
    if (i == n - 1) *count = pos[i] + (cand[i] != NONE ? 1 : 0);
  }
}

__global__ void iota_kernel(int64_t* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = i;
}

// Insertion of a sorted batch of new samples into the sorted sample set. Keys
// are distinct, so an entry's place in the merged order is its index plus the
// number of entries of the other array with a smaller key.
__device__ __forceinline__ int64_t count_below(const uint64_t* __restrict__ a, int64_t n, uint64_t k) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < k) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Main order: rows [0, n) of the arrays are sorted; rows [n, n + m) are new,
// nkey their keys sorted and row n + nperm[j] (nperm null: n + j) the data of
// nkey[j]. Output to o*.
__global__ void merge_samples_kernel(const uint64_t* __restrict__ key, const float* __restrict__ q,
                                     const float* __restrict__ L, const uint8_t* __restrict__ fa,
                                     const uint8_t* __restrict__ st, const int32_t* __restrict__ org, int64_t n,
                                     const uint64_t* __restrict__ nkey, const int64_t* __restrict__ nperm,
                                     int64_t m, uint64_t* okey, float* oq, float* oL, uint8_t* ofa, uint8_t* ost,
                                     int32_t* oorg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n + m; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t p, src;
    uint64_t k;
    if (i < n) {
      k = key[i];
      p = i + count_below(nkey, m, k);
      src = i;
    } else {
      int64_t j = i - n;
      k = nkey[j];
      p = j + count_below(key, n, k);
      src = n + (nperm ? nperm[j] : j);
    }
    okey[p] = k;
    oq[p] = q[src];
    oL[p] = L[src];
    ofa[2 * p] = fa[2 * src];
    ofa[2 * p + 1] = fa[2 * src + 1];
    ost[p] = st[src];
    if (org) oorg[p] = org[src];
  }
}

__global__ void fill_i32_kernel(int32_t* p, int64_t n, int32_t v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// A shifted-curve order (shifted key, length), sorted; new entries nskey
// (sorted) with lengths nL[nperm[j]].
__global__ void merge_order_kernel(const uint64_t* __restrict__ skey, const float* __restrict__ sL, int64_t n,
                                   const uint64_t* __restrict__ nskey, const int64_t* __restrict__ nperm,
                                   const float* __restrict__ nL, int64_t m, uint64_t* oskey, float* osL) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n + m; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) {
      int64_t p = i + count_below(nskey, m, skey[i]);
      oskey[p] = skey[i];
      osL[p] = sL[i];
    } else {
      int64_t j = i - n;
      int64_t p = j + count_below(skey, n, nskey[j]);
      oskey[p] = nskey[j];
      osL[p] = nL[nperm[j]];
    }
  }
}

// Outputs of samples traced in a separate batch (keys bkey[j], all present
// in the sorted set `key`) written to their places in the set.
__global__ void scatter_by_key_kernel(const uint64_t* __restrict__ bkey, int64_t m, const uint64_t* __restrict__ key,
                                      int64_t n, const float* __restrict__ q, const float* __restrict__ L,
                                      const uint8_t* __restrict__ fa, const uint8_t* __restrict__ st, float* oq,
                                      float* oL, uint8_t* ofa, uint8_t* ost) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = count_below(key, n, bkey[j]);
    if (p >= n || key[p] != bkey[j]) continue;  // not in the set (cannot happen)
    oq[p] = q[j];
    oL[p] = L[j];
    ofa[2 * p] = fa[2 * j];
    ofa[2 * p + 1] = fa[2 * j + 1];
    ost[p] = st[j];
  }
}

__global__ void gather_f_kernel(const int64_t* __restrict__ perm, int64_t n, const float* __restrict__ in,
                                float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[perm[i]];
}


// Converter: one thread per output cell.
__global__ void convert_kernel(const uint64_t* __restrict__ keys, const float* __restrict__ vals, int64_t n, int nd,
                               int bits, int d, int eo0, int eo1, int eo2, int log_interp, float* out) {
  int64_t N = (int64_t)eo0 * eo1 * eo2;
  uint64_t blk = 1ull << (nd * d);
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < N; o += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = o % eo0, rem = o / eo0;
    int64_t j = rem % eo1, k = rem / eo1;
    uint32_t c[3] = {(uint32_t)(i << d), (uint32_t)(j << d), (uint32_t)(k << d)};
    uint64_t k0 = (hilbert_key_dev(c, nd, bits) / blk) * blk;
    uint64_t k1 = k0 + blk;
    // lower bound of k0
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (keys[mid] < k0) lo = mid + 1; else hi = mid;
    }
    float res = __int_as_float(0x7fc00000);
    if (lo < n && keys[lo] < k1) {
      // maximum over the samples of the cell (NaNs ignored unless all NaN)
      for (int64_t s = lo; s < n && keys[s] < k1; ++s) {
        float v = vals[s];
        if (isnan(res) || v > res) res = isnan(v) ? res : v;
      }
    } else if (n > 0) {
      int64_t succ = lo, pred = lo - 1;
      if (succ >= n) {
        res = vals[pred];
      } else if (pred < 0) {
        res = vals[succ];
      } else {
        double kc = (double)k0 + 0.5 * (double)(blk - 1);
        double t = (kc - (double)keys[pred]) / ((double)keys[succ] - (double)keys[pred]);
        double a = vals[pred], b = vals[succ];
        if (log_interp)
          res = (float)exp10((1 - t) * log10(a) + t * log10(b));
        else
          res = (float)((1 - t) * a + t * b);
      }
    }
    out[o] = res;
  }
}

// Converter for an output lattice equal to the sample lattice (one lattice
// cell per output cell): same rule as convert_kernel, tiled along the curve.
// A block takes CK consecutive curve keys; its samples (and one neighbour on
// each side) are found from the chunk bounds (one binary search per chunk,
// all chunks in parallel, in chunk_bounds_kernel), staged in shared memory
// with their log10 values (FP64) and key-gap reciprocals, and each key is
// resolved there. Keys outside the extent are skipped. Q is interpolated in
// log10 in FP64 and the power evaluated as 2^(integer part) * 2^(fraction),
// the fraction by exp2f and the integer part exactly (ldexpf): a few FP32
// ulps, against one FP64 exp10 per empty cell.
constexpr int CK = 1024;
constexpr int CS = CK + 2;

__global__ void chunk_bounds_kernel(const uint64_t* __restrict__ keys, int64_t n, uint64_t nchunks,
                                    int64_t* __restrict__ start) {
  for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c <= nchunks; c += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k0 = c * CK;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (keys[mid] < k0) lo = mid + 1;
      else hi = mid;
    }
    start[c] = lo;
  }
}

__device__ __forceinline__ float pow10_of(double x) {
  if (!isfinite(x)) return (float)exp10(x);
  const double y = x * 3.321928094887362347870319429489390175864831393;  // log2(10)
  const double yi = floor(y);
  return ldexpf(exp2f((float)(y - yi)), (int)yi);
}

__global__ void __launch_bounds__(256) convert_tiled_kernel(const uint64_t* __restrict__ keys,
                                                            const float* __restrict__ vals, int64_t n, int nd,
                                                            int bits, int e0, int e1, int e2, int log_interp,
                                                            uint64_t nkeys, const int64_t* __restrict__ start,
                                                            float* out) {
  __shared__ uint64_t sk[CS];
  __shared__ float sv[CS];
  __shared__ double sl[CS];
  __shared__ double sinv[CS];
  for (uint64_t c0 = (uint64_t)blockIdx.x * CK; c0 < nkeys; c0 += (uint64_t)gridDim.x * CK) {
    const uint64_t c1 = c0 + CK < nkeys ? c0 + CK : nkeys;
    const uint64_t ci = c0 / CK;
    int64_t a = start[ci], b = start[ci + 1];
    if (a > 0) a -= 1;  // predecessor of the chunk
    if (b < n) b += 1;  // successor of the chunk
    const int cnt = (int)(b - a);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      sk[i] = keys[a + i];
      sv[i] = vals[a + i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      if (log_interp) sl[i] = log10((double)sv[i]);
      if (i + 1 < cnt) sinv[i] = 1.0 / (double)(sk[i + 1] - sk[i]);
    }
    __syncthreads();
    for (uint64_t k = c0 + threadIdx.x; k < c1; k += blockDim.x) {
      uint32_t c[3] = {0, 0, 0};
      hilbert_coords_dev(k, nd, bits, c);
      if ((int)c[0] >= e0 || (int)c[1] >= e1 || (nd == 3 && (int)c[2] >= e2)) continue;
      float res = __int_as_float(0x7fc00000);
      if (cnt > 0) {
        int lo = 0, hi = cnt;  // j: last staged sample with key <= k
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (sk[mid] <= k) lo = mid + 1;
          else hi = mid;
        }
        const int j = lo - 1;
        if (j >= 0 && sk[j] == k) {
          res = sv[j];
        } else if (j + 1 >= cnt) {
          res = sv[j];  // after the last sample
        } else if (j < 0) {
          res = sv[0];  // before the first sample
        } else {
          const double t = (double)(k - sk[j]) * sinv[j];
          if (log_interp)
            res = pow10_of((1 - t) * sl[j] + t * sl[j + 1]);
          else
            res = (float)((1 - t) * (double)sv[j] + t * (double)sv[j + 1]);
        }
      }
      out[(int64_t)c[0] + (int64_t)e0 * ((int64_t)c[1] + (int64_t)e1 * (int64_t)c[2])] = res;
    }
    __syncthreads();
  }
}

// Both grids of a refinement, Q (log10 interpolation) and L (linear), in one
// pass over the curve keys: convert_tiled_kernel's staging, Hilbert decodes
// and binary searches shared by the two value arrays, each resolved by the
// same rule.
__global__ void __launch_bounds__(256) convert_tiled_qL_kernel(const uint64_t* __restrict__ keys,
                                                               const float* __restrict__ qv,
                                                               const float* __restrict__ lv, int64_t n, int nd,
                                                               int bits, int e0, int e1, int e2, uint64_t nkeys,
                                                               const int64_t* __restrict__ start, float* qout,
                                                               float* lout) {
  __shared__ uint64_t sk[CS];
  __shared__ float sq[CS];
  __shared__ float sL[CS];
  __shared__ double sl[CS];
  __shared__ double sinv[CS];
  for (uint64_t c0 = (uint64_t)blockIdx.x * CK; c0 < nkeys; c0 += (uint64_t)gridDim.x * CK) {
    const uint64_t c1 = c0 + CK < nkeys ? c0 + CK : nkeys;
    const uint64_t ci = c0 / CK;
    int64_t a = start[ci], b = start[ci + 1];
    if (a > 0) a -= 1;  // predecessor of the chunk
    if (b < n) b += 1;  // successor of the chunk
    const int cnt = (int)(b - a);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      sk[i] = keys[a + i];
      sq[i] = qv[a + i];
      sL[i] = lv[a + i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      sl[i] = log10((double)sq[i]);
      if (i + 1 < cnt) sinv[i] = 1.0 / (double)(sk[i + 1] - sk[i]);
    }
    __syncthreads();
    for (uint64_t k = c0 + threadIdx.x; k < c1; k += blockDim.x) {
      uint32_t c[3] = {0, 0, 0};
      hilbert_coords_dev(k, nd, bits, c);
      if ((int)c[0] >= e0 || (int)c[1] >= e1 || (nd == 3 && (int)c[2] >= e2)) continue;
      float rq = __int_as_float(0x7fc00000), rl = rq;
      if (cnt > 0) {
        int lo = 0, hi = cnt;  // j: last staged sample with key <= k
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (sk[mid] <= k) lo = mid + 1;
          else hi = mid;
        }
        const int j = lo - 1;
        if (j >= 0 && sk[j] == k) {
          rq = sq[j];
          rl = sL[j];
        } else if (j + 1 >= cnt) {
          rq = sq[j];  // after the last sample
          rl = sL[j];
        } else if (j < 0) {
          rq = sq[0];  // before the first sample
          rl = sL[0];
        } else {
          const double t = (double)(k - sk[j]) * sinv[j];
          rq = pow10_of((1 - t) * sl[j] + t * sl[j + 1]);
          rl = (float)((1 - t) * (double)sL[j] + t * (double)sL[j + 1]);
        }
      }
      const int64_t o = (int64_t)c[0] + (int64_t)e0 * ((int64_t)c[1] + (int64_t)e1 * (int64_t)c[2]);
      qout[o] = rq;
      lout[o] = rl;
    }
    __syncthreads();
  }
}

int grid_for(int64_t n) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t b = (n + 255) / 256;
  if (b > (int64_t)sms * 16) b = (int64_t)sms * 16;
  return b < 1 ? 1 : (int)b;
}

// Scratch buffers of one refine call (stream-ordered allocations).
struct Scratch {
  std::vector<void*> bufs;
  cudaStream_t s;
  template <class T>
  int alloc(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = qsl::alloc_async((void**)&q, count * sizeof(T) + 16, s);
    if (e != cudaSuccess) {
      set_error("stream-ordered allocation of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
      return QSL_ENOMEM;
    }
    bufs.push_back(q);
    *p = (T*)q;
    return QSL_OK;
  }
  ~Scratch() {
    for (void* b : bufs) cudaFreeAsync(b, s);
  }
};

// Radix sort of (key, value) pairs on the low `bits` bits.
int sort_pairs(const uint64_t* kin, uint64_t* kout, const int64_t* vin, int64_t* vout, int64_t n, int bits,
               cudaStream_t s) {
  if (n <= 0) return QSL_OK;
  size_t tmp = 0;
  QSL_CHECK_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp, kin, kout, vin, vout, n, 0, bits, s));
  void* t = nullptr;
  QSL_CHECK_CUDA(qsl::alloc_async((void**)&t, tmp + 16, s));
  QSL_CHECK_CUDA(cub::DeviceRadixSort::SortPairs(t, tmp, kin, kout, vin, vout, n, 0, bits, s));
  QSL_CHECK_CUDA(cudaFreeAsync(t, s));
  return QSL_OK;
}

int exclusive_sum(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return QSL_OK;
  size_t tmp = 0;
  QSL_CHECK_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp, in, out, n, s));
  void* t = nullptr;
  QSL_CHECK_CUDA(qsl::alloc_async((void**)&t, tmp + 16, s));
  QSL_CHECK_CUDA(cub::DeviceScan::ExclusiveSum(t, tmp, in, out, n, s));
  QSL_CHECK_CUDA(cudaFreeAsync(t, s));
  return QSL_OK;
}

}  // namespace

int convert_device(const uint64_t* keys, const float* vals, int64_t n, int nd, int p, const int32_t* extent,
                   int out_order, int log_interp, float* out, cudaStream_t s) {
  int d = p - out_order;
  int eo[3] = {1, 1, 1};
  for (int a = 0; a < nd; ++a) eo[a] = extent[a] >> d;
  int64_t N = (int64_t)eo[0] * eo[1] * eo[2];
  if (N > 0 && d == 0) {
    const uint64_t nkeys = 1ull << (nd * p);
    int dev = 0, sms = 0;
    QSL_CHECK_CUDA(cudaGetDevice(&dev));
    QSL_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    uint64_t chunks = (nkeys + CK - 1) / CK;
    int64_t* start = nullptr;
    QSL_CHECK_CUDA(qsl::alloc_async((void**)&start, (chunks + 1) * sizeof(int64_t), s));
    chunk_bounds_kernel<<<grid_for((int64_t)chunks + 1), 256, 0, s>>>(keys, n, chunks, start);
    qsl::count_launch();
    QSL_CHECK_CUDA(cudaGetLastError());
    int blocks = chunks < (uint64_t)sms * 8 ? (int)chunks : sms * 8;
    convert_tiled_kernel<<<blocks, 256, 0, s>>>(keys, vals, n, nd, p, eo[0], eo[1], eo[2], log_interp, nkeys, start,
                                                out);
    qsl::count_launch();
    QSL_CHECK_CUDA(cudaGetLastError());
    QSL_CHECK_CUDA(cudaFreeAsync(start, s));
  } else if (N > 0) {
    convert_kernel<<<grid_for(N), 256, 0, s>>>(keys, vals, n, nd, p, d, eo[0], eo[1], eo[2], log_interp, out);
    qsl::count_launch();
    QSL_CHECK_CUDA(cudaGetLastError());
  }
  return QSL_OK;
}

// The refinement driver (device arrays). `smp` arrays are device pointers.
int refine_body(const qsl_field* f, const qsl_refine_spec* sp, const qsl_opts* o, qsl_samples* smp,
                float* q_grid, float* l_grid, int mem_proposal, cudaStream_t s);

// Event pairs of the last qsl_refine on this thread: [0] spans the call,
// then one pair per trace call (kind 0: coarse or proposal, 1: pass).
struct RefineClock {
  std::vector<cudaEvent_t> ev;  // pool, grown on demand, kept until exit
  std::vector<int> kind;
  std::vector<int64_t> lines;
  size_t used = 0;
  int iters = 0;
  static constexpr int kSnaps = 512;
  DeviceStats* snap = nullptr;  // device, one per trace call (the first kSnaps)
  int64_t* count_h = nullptr;   // pinned host word for the per-pass sample counts
  cudaStream_t stream = nullptr;
  bool valid = false;
  int device = -1;
  int take(cudaEvent_t* a, cudaEvent_t* b) {
    while (ev.size() < used + 2) {
      cudaEvent_t e;
      QSL_CHECK_CUDA(cudaEventCreate(&e));
      ev.push_back(e);
    }
    *a = ev[used];
    *b = ev[used + 1];
    used += 2;
    return QSL_OK;
  }
};
thread_local RefineClock g_rclock;

int refine_device(const qsl_field* f, const qsl_refine_spec* sp, const qsl_opts* o, qsl_samples* smp,
                  float* q_grid, float* l_grid, int mem_proposal, cudaStream_t s) {
  RefineClock& rk = g_rclock;
  {
    int dev = 0;
    QSL_CHECK_CUDA(cudaGetDevice(&dev));
    if (rk.device != dev) {
      // events and the snapshot buffer belong to a device: new ones for a new one
      rk.ev.clear();
      rk.snap = nullptr;
      rk.device = dev;
    }
    if (!rk.snap) QSL_CHECK_CUDA(cudaMalloc((void**)&rk.snap, sizeof(DeviceStats) * RefineClock::kSnaps));
    if (!rk.count_h) QSL_CHECK_CUDA(cudaMallocHost((void**)&rk.count_h, sizeof(int64_t)));
  }
  rk.used = 0;
  rk.kind.clear();
  rk.lines.clear();
  rk.iters = 0;
  rk.stream = s;
  rk.valid = false;
  cudaEvent_t call0, call1;
  {
    int r0 = rk.take(&call0, &call1);
    if (r0) return r0;
  }
  QSL_CHECK_CUDA(cudaEventRecord(call0, s));
  int rc_all = refine_body(f, sp, o, smp, q_grid, l_grid, mem_proposal, s);
  QSL_CHECK_CUDA(cudaEventRecord(call1, s));
  rk.iters = smp->iters;
  rk.valid = true;
  return rc_all;
}

// The sorted sample set sits in one of two sets of arrays (the caller's and a
// scratch set): each merge reads one and writes the other, and the caller's
// arrays receive the set once at the end if it ended in the scratch set.
struct SampleArrays {
  uint64_t* key;
  float* q;
  float* L;
  uint8_t* fa;
  uint8_t* st;
  int32_t* org;  // optional
};

int refine_body(const qsl_field* f, const qsl_refine_spec* sp, const qsl_opts* o, qsl_samples* smp,
                float* q_grid, float* l_grid, int mem_proposal, cudaStream_t s) {
  RefineClock& rk = g_rclock;
  int trace_kind = 0;  // 0 until the refinement iterations start
  const int nd = sp->ndim, p = sp->max_order, p0 = sp->coarse_order;
  const int R = 1 << (p - p0);
  int ext[3] = {1, 1, 1};
  for (int a = 0; a < nd; ++a) ext[a] = sp->extent[a] > 0 ? sp->extent[a] : (1 << p);
  Region reg;
  for (int a = 0; a < 3; ++a) {
    reg.lo[a] = 0;
    reg.hi[a] = a < nd ? (uint64_t)ext[a] : 1;
  }
  SeedSource src{};
  src.kind = nd == 2 ? SEEDS_KEYS2 : SEEDS_KEYS3;
  src.bits = p;
  for (int a = 0; a < 3; ++a) src.n[a] = ext[a];
  for (int k = 0; k < 3; ++k) {
    if (nd == 2) {
      src.c[k] = sp->center[k];
      src.u[k] = sp->u[k];
      src.v[k] = sp->v[k];
    } else {
      src.c[k] = sp->lo[k];
      src.u[k] = sp->hi[k];
    }
  }
  Scratch sc;
  sc.s = s;
  int64_t cap = smp->capacity;
  int64_t n = smp->count;
  int rc;
  int64_t* cnt = nullptr;        // device counter
  int64_t* cnt_h = rk.count_h;   // pinned host copy (kept per thread and device)
  if ((rc = sc.alloc(&cnt, 1))) return rc;
  int64_t traced = 0;
  bool cap_hit = false;

  // temporaries sized to the capacity
  uint64_t *kA = nullptr, *cand = nullptr, *sk = nullptr, *sk2 = nullptr;
  int64_t *perm = nullptr, *perm2 = nullptr, *flags = nullptr, *pos = nullptr;
  float *q2 = nullptr, *L2 = nullptr, *pvals = nullptr;
  uint8_t *fa2 = nullptr, *st2 = nullptr;
  int32_t* org2 = nullptr;
  if ((rc = sc.alloc(&kA, cap)) || (rc = sc.alloc(&cand, cap)) || (rc = sc.alloc(&sk, cap)) ||
      (rc = sc.alloc(&sk2, cap)) || (rc = sc.alloc(&perm, cap)) || (rc = sc.alloc(&perm2, cap)) ||
      (rc = sc.alloc(&flags, cap)) || (rc = sc.alloc(&pos, cap)) || (rc = sc.alloc(&q2, cap)) ||
      (rc = sc.alloc(&L2, cap)) || (rc = sc.alloc(&fa2, 2 * cap)) || (rc = sc.alloc(&st2, cap)))
    return rc;
  if (smp->origin && (rc = sc.alloc(&org2, cap))) return rc;
  const SampleArrays user{smp->key, smp->q, smp->length, smp->faces, smp->status, smp->origin};
  SampleArrays cur = user;                                // the set: rows [0, n) sorted, new rows after
  SampleArrays alt{kA, q2, L2, fa2, st2, smp->origin ? org2 : nullptr};  // the other array set

  // the criterion and the per-sample value it reads (L or Q)
  Criterion crit{sp->criterion, sp->tau, sp->q_threshold};
  auto crit_values = [&]() -> float* { return sp->criterion == QSL_REFINE_Q_THRESHOLD ? cur.q : cur.L; };

  // Shifted-curve orders (shifted key, criterion value) for the two alternating
  // shifts of pass B, built on first use and then kept sorted: before each use
  // the samples added since the last one are sorted and merged in at once, so
  // no pass re-sorts the set.
  const uint32_t half = 1u << (p - 1 >= 0 ? p - 1 : 0);
  const uint32_t dsh = (uint32_t)(R / 2 > 1 ? R / 2 : 1);
  const uint32_t shiftS[2] = {half + dsh, half - (dsh < half ? dsh : half)};
  uint64_t* ord_key[2] = {nullptr, nullptr};
  float* ord_L[2] = {nullptr, nullptr};
  uint64_t* ord_ktmp = nullptr;
  float* ord_Ltmp = nullptr;
  bool ord_built[2] = {false, false};
  int64_t ord_n[2] = {0, 0}, ord_mark[2] = {0, 0};  // entries; pass samples (pkeys) merged so far
  int64_t* nperm = nullptr;
  uint64_t* nkey = nullptr;
  if (sp->shift) {
    if ((rc = sc.alloc(&ord_key[0], cap)) || (rc = sc.alloc(&ord_key[1], cap)) || (rc = sc.alloc(&ord_L[0], cap)) ||
        (rc = sc.alloc(&ord_L[1], cap)) || (rc = sc.alloc(&ord_ktmp, cap)) || (rc = sc.alloc(&ord_Ltmp, cap)) ||
        (rc = sc.alloc(&pvals, cap)))
      return rc;
  }
  if ((rc = sc.alloc(&nperm, cap)) || (rc = sc.alloc(&nkey, cap))) return rc;

  // With the FLL-jump criterion the passes need lengths only: they trace in
  // length-only mode, and one launch after the last iteration traces every
  // pass sample with the deviation equations; its Q, L, end faces and status
  // (FP64 retrace above retrace_q included) replace the pass values, whose
  // lengths only decided the refinement. The decision traces take the paper's
  // Cash-Karp stepper across cells with the step cap pass_h_max (a step spans
  // several cells, where the cell-wise stepper lands on every face), or, on
  // request, the run's own integrator: only the cell-wise one keeps its length
  // bar without the deviation components, which hold the Cash-Karp stepper to
  // its tolerance across the kinks of the trilinear field.
  const bool fll_pass = sp->criterion == QSL_REFINE_FLL_JUMP && !o->length_only;
  qsl_opts o_len = *o;
  o_len.length_only = 1;
  bool decouple = false;
  if (fll_pass && sp->pass_stepper == QSL_PASS_CASH_KARP && f->geom == QSL_GEOM_CARTESIAN) {
    decouple = true;
    o_len.integrator = QSL_RKCK54;
    o_len.h_max = sp->pass_h_max > 0 ? sp->pass_h_max : 4.0;
  } else if (fll_pass && sp->pass_stepper == QSL_PASS_SAME) {
    decouple = o->integrator == QSL_DOPRI5_CELL && f->uniform;
  }
  uint64_t* pkeys = nullptr;  // keys of the pass samples in the order traced
  int64_t n_pass = 0;
  if ((rc = sc.alloc(&pkeys, cap))) return rc;

  // trace samples [off, off + m) of the current arrays (keys already written;
  // `sorted`: in key order) and merge them into the sorted set
  auto trace_and_merge = [&](int64_t off, int64_t m, bool sorted, int32_t pass_id) -> int {
    if (m <= 0) return QSL_OK;
    if (cur.org) {
      fill_i32_kernel<<<grid_for(m), 256, 0, s>>>(cur.org + off, m, pass_id);
      qsl::count_launch();
    }
    SeedSource s2 = src;
    s2.keys = cur.key + off;
    LineOutputs lo{};
    lo.q = cur.q + off;
    lo.length = cur.L + off;
    lo.faces = cur.fa + 2 * off;
    lo.status = cur.st + off;
    lo.q_form = o->q_form;
    lo.skip_open = o->skip_open;
    cudaEvent_t e0, e1;
    int r = rk.take(&e0, &e1);
    if (r) return r;
    QSL_CHECK_CUDA(cudaEventRecord(e0, s));
    const bool len_only = decouple && trace_kind == 1;
    r = run_lines(f, s2, m, len_only ? &o_len : o, lo, s);
    if (r) return r;
    QSL_CHECK_CUDA(cudaEventRecord(e1, s));
    if (trace_kind == 1) {
      QSL_CHECK_CUDA(
          cudaMemcpyAsync(pkeys + n_pass, cur.key + off, m * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
      n_pass += m;
    }
    if (rk.kind.size() < (size_t)RefineClock::kSnaps)
      QSL_CHECK_CUDA(cudaMemcpyAsync(rk.snap + rk.kind.size(), last_run_stats_dev(), sizeof(DeviceStats),
                                     cudaMemcpyDeviceToDevice, s));
    rk.kind.push_back(trace_kind);
    rk.lines.push_back(m);
    traced += m;
    // the batch in key order
    const uint64_t* bkey = cur.key + off;
    const int64_t* bperm = nullptr;
    if (!sorted) {
      iota_kernel<<<grid_for(m), 256, 0, s>>>(perm, m);
      qsl::count_launch();
      if ((r = sort_pairs(cur.key + off, nkey, perm, nperm, m, nd * p, s))) return r;
      bkey = nkey;
      bperm = nperm;
    }
    int64_t tot = off + m;
    merge_samples_kernel<<<grid_for(tot), 256, 0, s>>>(cur.key, cur.q, cur.L, cur.fa, cur.st, cur.org, off, bkey,
                                                        bperm, m, alt.key, alt.q, alt.L, alt.fa, alt.st, alt.org);
    qsl::count_launch();
    QSL_CHECK_CUDA(cudaGetLastError());
    std::swap(cur, alt);
    return QSL_OK;
  };

  // compact candidates cand[0..m) (flags[i] = cand[i] is one) into the rows
  // after the set, returns the number added
  auto compact = [&](int64_t m, int64_t* added) -> int {
    *added = 0;
    if (m <= 0) return QSL_OK;
    int r = exclusive_sum(flags, pos, m, s);
    if (r) return r;
    cand_scatter_kernel<<<grid_for(m), 256, 0, s>>>(cand, pos, m, cap - n, cur.key + n, cnt);
    qsl::count_launch();
    QSL_CHECK_CUDA(cudaGetLastError());
    QSL_CHECK_CUDA(cudaMemcpyAsync(cnt_h, cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    QSL_CHECK_CUDA(cudaStreamSynchronize(s));
    int64_t a = *cnt_h;
    if (a > cap - n) {
      a = cap - n;
      cap_hit = true;
    }
    *added = a;
    return QSL_OK;
  };

  if (n == 0) {
    // coarse pass
    int nc[3] = {1, 1, 1};
    for (int a = 0; a < nd; ++a) nc[a] = ext[a] / R;
    int64_t m = (int64_t)nc[0] * nc[1] * nc[2];
    if (m > cap) {
      set_error("capacity %lld below the %lld coarse samples", (long long)cap, (long long)m);
      return QSL_ECAPACITY;
    }
    coarse_keys_kernel<<<grid_for(m), 256, 0, s>>>(m, nd, p, R, nc[0], nc[1], cur.key);
    qsl::count_launch();
    QSL_CHECK_CUDA(cudaGetLastError());
    // trace in curve order (neighbouring seeds on neighbouring lanes)
    iota_kernel<<<grid_for(m), 256, 0, s>>>(perm, m);
    qsl::count_launch();
    if ((rc = sort_pairs(cur.key, nkey, perm, perm2, m, nd * p, s))) return rc;
    QSL_CHECK_CUDA(cudaMemcpyAsync(cur.key, nkey, m * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    if ((rc = trace_and_merge(0, m, true, 0))) return rc;
    n = m;
  }
  // optional proposal (fresh runs and resumed ones): every effective cell of
  // the flagged coarse cells that is not a sample yet is traced, before the
  // FLL-jump iterations, which then continue as the fallback criterion
  if (sp->proposal) {
    int nc[3] = {1, 1, 1};
    for (int a = 0; a < nd; ++a) nc[a] = ext[a] / R;
    int64_t m = (int64_t)nc[0] * nc[1] * nc[2];
    const uint8_t* mask = sp->proposal;
    uint8_t* mask_dev = nullptr;
    if (mem_proposal == QSL_MEM_HOST) {
      if ((rc = sc.alloc(&mask_dev, m))) return rc;
      QSL_CHECK_CUDA(cudaMemcpyAsync(mask_dev, mask, m, cudaMemcpyHostToDevice, s));
      mask = mask_dev;
    }
    int64_t* cells = nullptr;
    if ((rc = sc.alloc(&cells, m))) return rc;
    QSL_CHECK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int64_t), s));
    mask_cells_kernel<<<grid_for(m), 256, 0, s>>>(mask, m, cells, cnt);
    qsl::count_launch();
    QSL_CHECK_CUDA(cudaMemcpyAsync(cnt_h, cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    QSL_CHECK_CUDA(cudaStreamSynchronize(s));
    int64_t ncells = *cnt_h;
    const int pst = sp->proposal_stride > 1 ? sp->proposal_stride : 1;
    int64_t per = 1;
    for (int a = 0; a < nd; ++a) per *= R / pst;
    int64_t want = ncells * per;
    if (want > cap - n) {
      set_error("capacity too small for the proposal (up to %lld more samples)", (long long)want);
      return QSL_ECAPACITY;
    }
    if (want > 0) {
      int64_t* ncd = nullptr;
      if ((rc = sc.alloc(&ncd, 1))) return rc;
      QSL_CHECK_CUDA(cudaMemcpyAsync(ncd, cnt, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
      QSL_CHECK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int64_t), s));
      proposal_keys_kernel<<<grid_for(want), 256, 0, s>>>(cells, ncd, nd, p, R, pst, nc[0], nc[1], cur.key, n,
                                                            cur.key + n, cnt);
      qsl::count_launch();
      QSL_CHECK_CUDA(cudaGetLastError());
      QSL_CHECK_CUDA(cudaMemcpyAsync(cnt_h, cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      QSL_CHECK_CUDA(cudaStreamSynchronize(s));
      int64_t got = *cnt_h;
      if (got > 0) {
        // trace the new cells in curve order (neighbouring seeds on neighbouring lanes)
        iota_kernel<<<grid_for(got), 256, 0, s>>>(perm, got);
        qsl::count_launch();
        if ((rc = sort_pairs(cur.key + n, nkey, perm, perm2, got, nd * p, s))) return rc;
        QSL_CHECK_CUDA(cudaMemcpyAsync(cur.key + n, nkey, got * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        if ((rc = trace_and_merge(n, got, true, 0))) return rc;
        n += got;
      }
    }
  }

  int it = 0;
  trace_kind = 1;
  for (; it < sp->max_iters && !cap_hit; ++it) {
    int64_t added_total = 0, added = 0;
    // (A) along the curve (candidates come out in key order)
    if (n > 1) {
      flag_pairs_kernel<<<grid_for(n - 1), 256, 0, s>>>(cur.key, crit_values(), n, crit, nd, p, reg, cand, flags);
      qsl::count_launch();
      QSL_CHECK_CUDA(cudaGetLastError());
      if ((rc = compact(n - 1, &added))) return rc;
      if ((rc = trace_and_merge(n, added, true, 2 * it + 1))) return rc;
      n += added;
      added_total += added;
    }
    // (B) along the shifted curve
    if (sp->shift && n > 1 && !cap_hit) {
      const int b = it % 2;
      const uint32_t S = shiftS[b];
      if (!ord_built[b]) {
        shift_keys_kernel<<<grid_for(n), 256, 0, s>>>(cur.key, n, nd, p, S, sk, perm);
        qsl::count_launch();
        QSL_CHECK_CUDA(cudaGetLastError());
        if ((rc = sort_pairs(sk, ord_key[b], perm, perm2, n, nd * (p + 1), s))) return rc;
        gather_f_kernel<<<grid_for(n), 256, 0, s>>>(perm2, n, crit_values(), ord_L[b]);
        qsl::count_launch();
        QSL_CHECK_CUDA(cudaGetLastError());
        ord_built[b] = true;
        ord_n[b] = n;
        ord_mark[b] = n_pass;
      } else if (ord_mark[b] < n_pass) {
        // the pass samples added since this order's last use, at once
        const int64_t m2 = n_pass - ord_mark[b];
        shift_lookup_kernel<<<grid_for(m2), 256, 0, s>>>(pkeys + ord_mark[b], m2, nd, p, S, cur.key, n,
                                                          crit_values(), sk, pvals, perm);
        qsl::count_launch();
        QSL_CHECK_CUDA(cudaGetLastError());
        if ((rc = sort_pairs(sk, sk2, perm, perm2, m2, nd * (p + 1), s))) return rc;
        merge_order_kernel<<<grid_for(ord_n[b] + m2), 256, 0, s>>>(ord_key[b], ord_L[b], ord_n[b], sk2, perm2,
                                                                     pvals, m2, ord_ktmp, ord_Ltmp);
        qsl::count_launch();
        QSL_CHECK_CUDA(cudaGetLastError());
        std::swap(ord_key[b], ord_ktmp);
        std::swap(ord_L[b], ord_Ltmp);
        ord_n[b] += m2;
        ord_mark[b] = n_pass;
      }
      if (ord_n[b] != n) {
        set_error("internal: shifted order holds %lld of %lld samples", (long long)ord_n[b], (long long)n);
        return QSL_ECUDA;
      }
      Region sreg;
      for (int a = 0; a < 3; ++a) {
        sreg.lo[a] = reg.lo[a] + (a < nd ? S : 0);
        sreg.hi[a] = reg.hi[a] + (a < nd ? S : 0);
      }
      flag_shifted_kernel<<<grid_for(n - 1), 256, 0, s>>>(ord_key[b], ord_L[b], n, crit, nd, p, S, sreg, cand,
                                                           flags);
      qsl::count_launch();
      QSL_CHECK_CUDA(cudaGetLastError());
      if ((rc = compact(n - 1, &added))) return rc;
      if ((rc = trace_and_merge(n, added, false, 2 * it + 2))) return rc;
      n += added;
      added_total += added;
    }
    if (added_total == 0) break;
  }
  if (decouple && n_pass > 0) {
    // Q of every pass sample (keys sorted first: neighbouring seeds on
    // neighbouring lanes), then scattered to its place in the sorted set
    float *q_s = nullptr, *L_s = nullptr;
    uint8_t *fa_s = nullptr, *st_s = nullptr;
    if ((rc = sc.alloc(&q_s, n_pass)) || (rc = sc.alloc(&L_s, n_pass)) || (rc = sc.alloc(&fa_s, 2 * n_pass)) ||
        (rc = sc.alloc(&st_s, n_pass)))
      return rc;
    iota_kernel<<<grid_for(n_pass), 256, 0, s>>>(perm, n_pass);
    qsl::count_launch();
    if ((rc = sort_pairs(pkeys, nkey, perm, nperm, n_pass, nd * p, s))) return rc;
    SeedSource s3 = src;
    s3.keys = nkey;
    LineOutputs lo{};
    lo.q = q_s;
    lo.length = L_s;
    lo.faces = fa_s;
    lo.status = st_s;
    lo.q_form = o->q_form;
    lo.skip_open = o->skip_open;
    cudaEvent_t e0, e1;
    if ((rc = rk.take(&e0, &e1))) return rc;
    QSL_CHECK_CUDA(cudaEventRecord(e0, s));
    if ((rc = run_lines(f, s3, n_pass, o, lo, s))) return rc;
    QSL_CHECK_CUDA(cudaEventRecord(e1, s));
    if (rk.kind.size() < (size_t)RefineClock::kSnaps)
      QSL_CHECK_CUDA(cudaMemcpyAsync(rk.snap + rk.kind.size(), last_run_stats_dev(), sizeof(DeviceStats),
                                     cudaMemcpyDeviceToDevice, s));
    rk.kind.push_back(2);
    rk.lines.push_back(n_pass);
    scatter_by_key_kernel<<<grid_for(n_pass), 256, 0, s>>>(nkey, n_pass, cur.key, n, q_s, L_s, fa_s, st_s, cur.q,
                                                            cur.L, cur.fa, cur.st);
    qsl::count_launch();
    QSL_CHECK_CUDA(cudaGetLastError());
  }
  if (cur.key != user.key && n > 0) {
    // the set ended in the scratch arrays
    QSL_CHECK_CUDA(cudaMemcpyAsync(user.key, cur.key, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    QSL_CHECK_CUDA(cudaMemcpyAsync(user.q, cur.q, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    QSL_CHECK_CUDA(cudaMemcpyAsync(user.L, cur.L, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    QSL_CHECK_CUDA(cudaMemcpyAsync(user.fa, cur.fa, 2 * n, cudaMemcpyDeviceToDevice, s));
    QSL_CHECK_CUDA(cudaMemcpyAsync(user.st, cur.st, n, cudaMemcpyDeviceToDevice, s));
    if (user.org) QSL_CHECK_CUDA(cudaMemcpyAsync(user.org, cur.org, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  }
  smp->count = n;
  smp->iters = it;
  smp->traced = (int32_t)(traced & 0x7fffffff);
  int out_order = sp->out_order > 0 ? sp->out_order : p;
  if (q_grid && l_grid && out_order == p && n > 0) {
    // both grids in one pass over the curve keys
    int eo[3] = {1, 1, 1};
    for (int a = 0; a < nd; ++a) eo[a] = ext[a];
    const uint64_t nkeys = 1ull << (nd * p);
    const uint64_t chunks = (nkeys + CK - 1) / CK;
    int64_t* start = nullptr;
    if ((rc = sc.alloc(&start, chunks + 1))) return rc;
    chunk_bounds_kernel<<<grid_for((int64_t)chunks + 1), 256, 0, s>>>(user.key, n, chunks, start);
    qsl::count_launch();
    int dev = 0, sms = 0;
    QSL_CHECK_CUDA(cudaGetDevice(&dev));
    QSL_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = chunks < (uint64_t)sms * 8 ? (int)chunks : sms * 8;
    convert_tiled_qL_kernel<<<blocks, 256, 0, s>>>(user.key, user.q, user.L, n, nd, p, eo[0], eo[1], eo[2], nkeys,
                                                   start, q_grid, l_grid);
    qsl::count_launch();
    QSL_CHECK_CUDA(cudaGetLastError());
  } else {
    if (q_grid && (rc = convert_device(user.key, user.q, n, nd, p, ext, out_order, 1, q_grid, s))) return rc;
    if (l_grid && (rc = convert_device(user.key, user.L, n, nd, p, ext, out_order, 0, l_grid, s))) return rc;
  }
  if (cap_hit) {
    set_error("sample capacity %lld reached", (long long)cap);
    return QSL_ECAPACITY;
  }
  return QSL_OK;
}

}  // namespace qsl

using namespace qsl;

extern "C" {

int qsl_last_refine_stats(qsl_refine_stats* out) {
  if (!out) {
    set_error("out is NULL");
    return QSL_EINVAL;
  }
  memset(out, 0, sizeof(*out));
  RefineClock& rk = g_rclock;
  if (!rk.valid) {
    set_error("no qsl_refine on this thread yet");
    return QSL_EINVAL;
  }
  QSL_CHECK_CUDA(cudaStreamSynchronize(rk.stream));
  float t = 0;
  QSL_CHECK_CUDA(cudaEventElapsedTime(&t, rk.ev[0], rk.ev[1]));
  out->total_ms = t;
  for (size_t i = 0; i < rk.kind.size(); ++i) {
    QSL_CHECK_CUDA(cudaEventElapsedTime(&t, rk.ev[2 + 2 * i], rk.ev[3 + 2 * i]));
    if (rk.kind[i] == 0) {
      out->coarse_ms += t;
      out->coarse_lines += rk.lines[i];
    } else if (rk.kind[i] == 1) {
      out->passes_ms += t;
      out->pass_lines += rk.lines[i];
      out->passes += 1;
    } else {
      out->deferred_ms += t;
    }
  }
  size_t ns = rk.kind.size() < (size_t)RefineClock::kSnaps ? rk.kind.size() : (size_t)RefineClock::kSnaps;
  std::vector<DeviceStats> h(ns);
  if (ns) QSL_CHECK_CUDA(cudaMemcpy(h.data(), rk.snap, sizeof(DeviceStats) * ns, cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < ns; ++i) {
    if (rk.kind[i] == 0) {
      out->coarse_stage_evals += (int64_t)h[i].stage_evals;
      out->coarse_landings += (int64_t)h[i].landing;
    } else if (rk.kind[i] == 1) {
      out->pass_stage_evals += (int64_t)h[i].stage_evals;
      out->pass_landings += (int64_t)h[i].landing;
    } else {
      out->deferred_stage_evals += (int64_t)h[i].stage_evals;
      out->deferred_landings += (int64_t)h[i].landing;
    }
  }
  out->iters = rk.iters;
  return QSL_OK;
}

int qsl_hilbert_encode(const uint32_t* coords, int64_t n, int ndim, int bits, uint64_t* keys, int mem,
                       void* stream_) {
  cudaStream_t s = (cudaStream_t)stream_;
  if ((ndim != 2 && ndim != 3) || bits < 0 || ndim * bits > 63 || n < 0) {
    set_error("bad ndim/bits/n");
    return QSL_EINVAL;
  }
  if (n == 0) return QSL_OK;
  if (!coords || !keys) {
    set_error("NULL array");
    return QSL_EINVAL;
  }
  const uint32_t* c = coords;
  uint64_t* k = keys;
  if (mem == QSL_MEM_HOST) {
    QSL_CHECK_CUDA(qsl::alloc_async((void**)&c, n * ndim * 4, s));
    QSL_CHECK_CUDA(qsl::alloc_async((void**)&k, n * 8, s));
    QSL_CHECK_CUDA(cudaMemcpyAsync((void*)c, coords, n * ndim * 4, cudaMemcpyHostToDevice, s));
  }
  encode_kernel<<<grid_for(n), 256, 0, s>>>(c, n, ndim, bits, k);
  qsl::count_launch();
  QSL_CHECK_CUDA(cudaGetLastError());
  if (mem == QSL_MEM_HOST) {
    QSL_CHECK_CUDA(cudaMemcpyAsync(keys, k, n * 8, cudaMemcpyDeviceToHost, s));
    QSL_CHECK_CUDA(cudaFreeAsync((void*)c, s));
    QSL_CHECK_CUDA(cudaFreeAsync(k, s));
    QSL_CHECK_CUDA(cudaStreamSynchronize(s));
  }
  return QSL_OK;
}

int qsl_hilbert_decode(const uint64_t* keys, int64_t n, int ndim, int bits, uint32_t* coords, int mem,
                       void* stream_) {
  cudaStream_t s = (cudaStream_t)stream_;
  if ((ndim != 2 && ndim != 3) || bits < 0 || ndim * bits > 63 || n < 0) {
    set_error("bad ndim/bits/n");
    return QSL_EINVAL;
  }
  if (n == 0) return QSL_OK;
  if (!coords || !keys) {
    set_error("NULL array");
    return QSL_EINVAL;
  }
  const uint64_t* k = keys;
  uint32_t* c = coords;
  if (mem == QSL_MEM_HOST) {
    QSL_CHECK_CUDA(qsl::alloc_async((void**)&k, n * 8, s));
    QSL_CHECK_CUDA(qsl::alloc_async((void**)&c, n * ndim * 4, s));
    QSL_CHECK_CUDA(cudaMemcpyAsync((void*)k, keys, n * 8, cudaMemcpyHostToDevice, s));
  }
  decode_kernel<<<grid_for(n), 256, 0, s>>>(k, n, ndim, bits, c);
  qsl::count_launch();
  QSL_CHECK_CUDA(cudaGetLastError());
  if (mem == QSL_MEM_HOST) {
    QSL_CHECK_CUDA(cudaMemcpyAsync(coords, c, n * ndim * 4, cudaMemcpyDeviceToHost, s));
    QSL_CHECK_CUDA(cudaFreeAsync((void*)k, s));
    QSL_CHECK_CUDA(cudaFreeAsync(c, s));
    QSL_CHECK_CUDA(cudaStreamSynchronize(s));
  }
  return QSL_OK;
}

int qsl_convert(const uint64_t* keys, const float* vals, int64_t n, int ndim, int max_order, const int32_t* extent,
                int out_order, int log_interp, float* out, int mem, void* stream_) {
  cudaStream_t s = (cudaStream_t)stream_;
  if ((ndim != 2 && ndim != 3) || max_order < 0 || ndim * max_order > 63 || out_order < 0 ||
      out_order > max_order || n < 0 || !extent || !out || (n > 0 && (!keys || !vals))) {
    set_error("bad converter arguments");
    return QSL_EINVAL;
  }
  int d = max_order - out_order;
  int64_t N = 1;
  for (int a = 0; a < ndim; ++a) {
    if (extent[a] < 1 || extent[a] > (1 << max_order) || (extent[a] & ((1 << d) - 1))) {
      set_error("extent[%d] must be in 1..2^max_order and a multiple of 2^(max_order-out_order)", a);
      return QSL_EINVAL;
    }
    N *= extent[a] >> d;
  }
  if (mem == QSL_MEM_DEVICE) return convert_device(keys, vals, n, ndim, max_order, extent, out_order, log_interp, out, s);
  uint64_t* k = nullptr;
  float *v = nullptr, *o = nullptr;
  QSL_CHECK_CUDA(qsl::alloc_async((void**)&k, n * 8 + 8, s));
  QSL_CHECK_CUDA(qsl::alloc_async((void**)&v, n * 4 + 4, s));
  QSL_CHECK_CUDA(qsl::alloc_async((void**)&o, N * 4, s));
  if (n) {
    QSL_CHECK_CUDA(cudaMemcpyAsync(k, keys, n * 8, cudaMemcpyHostToDevice, s));
    QSL_CHECK_CUDA(cudaMemcpyAsync(v, vals, n * 4, cudaMemcpyHostToDevice, s));
  }
  int rc = convert_device(k, v, n, ndim, max_order, extent, out_order, log_interp, o, s);
  if (rc) return rc;
  QSL_CHECK_CUDA(cudaMemcpyAsync(out, o, N * 4, cudaMemcpyDeviceToHost, s));
  QSL_CHECK_CUDA(cudaFreeAsync(k, s));
  QSL_CHECK_CUDA(cudaFreeAsync(v, s));
  QSL_CHECK_CUDA(cudaFreeAsync(o, s));
  QSL_CHECK_CUDA(cudaStreamSynchronize(s));
  return QSL_OK;
}

int qsl_refine(const qsl_field* f, const qsl_refine_spec* sp, const qsl_opts* o, qsl_samples* smp, float* q_grid,
               float* l_grid, int mem, void* stream_) {
  cudaStream_t s = (cudaStream_t)stream_;
  if (!f || !sp || !o || !smp) {
    set_error("NULL argument");
    return QSL_EINVAL;
  }
  if (sp->ndim != 2 && sp->ndim != 3) {
    set_error("ndim must be 2 or 3");
    return QSL_EINVAL;
  }
  int nd = sp->ndim, p = sp->max_order, p0 = sp->coarse_order;
  if (p0 < 0 || p < p0 || nd * (p + 1) > 63 || p > 30) {
    set_error("need 0 <= coarse_order <= max_order and ndim * (max_order + 1) <= 63");
    return QSL_EINVAL;
  }
  if (sp->criterion != QSL_REFINE_FLL_JUMP && sp->criterion != QSL_REFINE_Q_THRESHOLD) {
    set_error("criterion must be QSL_REFINE_FLL_JUMP or QSL_REFINE_Q_THRESHOLD");
    return QSL_EINVAL;
  }
  {
    const int pst = sp->proposal_stride;
    const int Rr = 1 << (sp->max_order - sp->coarse_order);
    if (pst < 0 || pst > Rr || (pst > 1 && (pst & (pst - 1)))) {
      set_error("proposal_stride must be 0, 1 or a power of two <= 2^(max_order - coarse_order)");
      return QSL_EINVAL;
    }
  }
  if (sp->pass_stepper < QSL_PASS_CASH_KARP || sp->pass_stepper > QSL_PASS_FULL ||
      !(sp->pass_h_max >= 0.0 && sp->pass_h_max < 1e6)) {
    set_error("pass_stepper must be QSL_PASS_CASH_KARP, QSL_PASS_SAME or QSL_PASS_FULL and 0 <= pass_h_max < 1e6");
    return QSL_EINVAL;
  }
  int R = 1 << (p - p0);
  for (int a = 0; a < nd; ++a) {
    int e = sp->extent[a] > 0 ? sp->extent[a] : (1 << p);
    if (e > (1 << p) || e % R) {
      set_error("extent[%d] = %d must be <= 2^max_order and a multiple of 2^(max_order - coarse_order)", a, e);
      return QSL_EINVAL;
    }
  }
  int oo = sp->out_order > 0 ? sp->out_order : p;
  if (oo > p) {
    set_error("out_order above max_order");
    return QSL_EINVAL;
  }
  if (smp->capacity < 1 || smp->count < 0 || smp->count > smp->capacity || !smp->key || !smp->q || !smp->length) {
    set_error("bad samples (capacity/count/arrays)");
    return QSL_EINVAL;
  }
  if (sp->max_iters < 0) {
    set_error("max_iters must be >= 0");
    return QSL_EINVAL;
  }
  if (mem == QSL_MEM_DEVICE) {
    // faces/status are optional: give the refinement loop scratch ones
    qsl_samples d = *smp;
    void* sf = nullptr;
    void* ss = nullptr;
    if (!d.faces) {
      QSL_CHECK_CUDA(qsl::alloc_async((void**)&sf, 2 * d.capacity, s));
      d.faces = (uint8_t*)sf;
    }
    if (!d.status) {
      QSL_CHECK_CUDA(qsl::alloc_async((void**)&ss, d.capacity, s));
      d.status = (uint8_t*)ss;
    }
    int rc = refine_device(f, sp, o, &d, q_grid, l_grid, QSL_MEM_DEVICE, s);
    smp->count = d.count;
    smp->iters = d.iters;
    smp->traced = d.traced;
    if (sf) cudaFreeAsync(sf, s);
    if (ss) cudaFreeAsync(ss, s);
    return rc;
  }
  if (mem != QSL_MEM_HOST) {
    set_error("bad mem %d", mem);
    return QSL_EINVAL;
  }
  int64_t cap = smp->capacity;
  qsl_samples d = *smp;
  QSL_CHECK_CUDA(qsl::alloc_async((void**)&d.key, cap * 8, s));
  QSL_CHECK_CUDA(qsl::alloc_async((void**)&d.q, cap * 4, s));
  QSL_CHECK_CUDA(qsl::alloc_async((void**)&d.length, cap * 4, s));
  QSL_CHECK_CUDA(qsl::alloc_async((void**)&d.faces, cap * 2, s));
  QSL_CHECK_CUDA(qsl::alloc_async((void**)&d.status, cap, s));
  int64_t c0 = smp->count;
  if (c0) {
    QSL_CHECK_CUDA(cudaMemcpyAsync(d.key, smp->key, c0 * 8, cudaMemcpyHostToDevice, s));
    QSL_CHECK_CUDA(cudaMemcpyAsync(d.q, smp->q, c0 * 4, cudaMemcpyHostToDevice, s));
    QSL_CHECK_CUDA(cudaMemcpyAsync(d.length, smp->length, c0 * 4, cudaMemcpyHostToDevice, s));
    if (smp->faces) QSL_CHECK_CUDA(cudaMemcpyAsync(d.faces, smp->faces, c0 * 2, cudaMemcpyHostToDevice, s));
    else QSL_CHECK_CUDA(cudaMemsetAsync(d.faces, 255, c0 * 2, s));
    if (smp->status) QSL_CHECK_CUDA(cudaMemcpyAsync(d.status, smp->status, c0, cudaMemcpyHostToDevice, s));
    else QSL_CHECK_CUDA(cudaMemsetAsync(d.status, 0, c0, s));
  }
  if (smp->origin) {
    QSL_CHECK_CUDA(qsl::alloc_async((void**)&d.origin, cap * 4, s));
    if (c0) QSL_CHECK_CUDA(cudaMemcpyAsync(d.origin, smp->origin, c0 * 4, cudaMemcpyHostToDevice, s));
  }
  int ext[3] = {1, 1, 1};
  for (int a = 0; a < nd; ++a) ext[a] = sp->extent[a] > 0 ? sp->extent[a] : (1 << p);
  int dd = p - oo;
  int64_t N = 1;
  for (int a = 0; a < nd; ++a) N *= ext[a] >> dd;
  float *qg = nullptr, *lg = nullptr;
  if (q_grid) QSL_CHECK_CUDA(qsl::alloc_async((void**)&qg, N * 4, s));
  if (l_grid) QSL_CHECK_CUDA(qsl::alloc_async((void**)&lg, N * 4, s));
  int rc = refine_device(f, sp, o, &d, qg, lg, QSL_MEM_HOST, s);
  if (rc == QSL_OK || rc == QSL_ECAPACITY) {
    int64_t n = d.count;
    if (n) {
      QSL_CHECK_CUDA(cudaMemcpyAsync(smp->key, d.key, n * 8, cudaMemcpyDeviceToHost, s));
      QSL_CHECK_CUDA(cudaMemcpyAsync(smp->q, d.q, n * 4, cudaMemcpyDeviceToHost, s));
      QSL_CHECK_CUDA(cudaMemcpyAsync(smp->length, d.length, n * 4, cudaMemcpyDeviceToHost, s));
      if (smp->faces) QSL_CHECK_CUDA(cudaMemcpyAsync(smp->faces, d.faces, n * 2, cudaMemcpyDeviceToHost, s));
      if (smp->status) QSL_CHECK_CUDA(cudaMemcpyAsync(smp->status, d.status, n, cudaMemcpyDeviceToHost, s));
      if (smp->origin) QSL_CHECK_CUDA(cudaMemcpyAsync(smp->origin, d.origin, n * 4, cudaMemcpyDeviceToHost, s));
    }
    if (qg) QSL_CHECK_CUDA(cudaMemcpyAsync(q_grid, qg, N * 4, cudaMemcpyDeviceToHost, s));
    if (lg) QSL_CHECK_CUDA(cudaMemcpyAsync(l_grid, lg, N * 4, cudaMemcpyDeviceToHost, s));
    smp->count = d.count;
    smp->iters = d.iters;
    smp->traced = d.traced;
  }
  cudaFreeAsync(d.key, s);
  cudaFreeAsync(d.q, s);
  cudaFreeAsync(d.length, s);
  cudaFreeAsync(d.faces, s);
  cudaFreeAsync(d.status, s);
  if (d.origin) cudaFreeAsync(d.origin, s);
  if (qg) cudaFreeAsync(qg, s);
  if (lg) cudaFreeAsync(lg, s);
  cudaStreamSynchronize(s);
  return rc;
}

}  // extern "C"
