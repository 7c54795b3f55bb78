// Corner queries and marching cubes in the predicted active cells (Sec. IV-D, last paragraph), the
// float32 point evaluation of the MLP, and the library's own marching-cubes case table.
#include "internal.cuh"
#include "linearise.cuh"

#include <algorithm>
#include <cstring>
#include <mutex>

namespace isx {

// ---- case table ----------------------------------------------------------------------------------
// Generated on the host from the rules stated in isx.h / the mesh module: inside = value < iso;
// faces with two crossings get one segment, faces with four get one segment around each inside
// corner; segments are directed with the face's inside corners on their right seen from outside;
// the segments chain into loops, fanned from their smallest edge number.
namespace {

// local edge number of the edge along `axis` whose other two axes (ascending) take bits b_lo, b_hi
int edge_number(int axis, int b_lo, int b_hi) { return 4 * axis + b_lo + 2 * b_hi; }

struct FaceEdge {
  int id;
  double u, v;   // midpoint in the face's (p, q) coordinates
  int c0, c1;    // its two corners (cube corner numbers)
};

int corner_of(int axis_a, int side, int p, int q, int bp, int bq) {
  int bits[3];
  bits[axis_a] = side;
  bits[p] = bp;
  bits[q] = bq;
  return bits[0] | (bits[1] << 1) | (bits[2] << 2);
}

void build_case(int cs, int8_t* ntri, int8_t* tris) {
  auto inside = [&](int c) { return (cs >> c) & 1; };
  int next[12];
  for (int e = 0; e < 12; ++e) next[e] = -1;
  bool crossing[12] = {};
  for (int a = 0; a < 3; ++a) {
    int p = a == 0 ? 1 : 0, q = a == 2 ? 1 : 2;
    // orientation of (p, q) seen from outside the face (+1: counter-clockwise)
    bool cyclic = ((p + 1) % 3 == q);
    for (int side = 0; side < 2; ++side) {
      int orient = (cyclic ? 1 : -1) * (side ? 1 : -1);
      // the four edges of this face
      FaceEdge fe[4];
      int nf = 0;
      for (int bq = 0; bq < 2; ++bq) {   // edges along p at q = bq
        int lo = std::min(a, q) == a ? side : bq, hi = std::min(a, q) == a ? bq : side;
        fe[nf++] = {edge_number(p, lo, hi), 0.5, (double)bq, corner_of(a, side, p, q, 0, bq),
                    corner_of(a, side, p, q, 1, bq)};
      }
      for (int bp = 0; bp < 2; ++bp) {   // edges along q at p = bp
        int lo = std::min(a, p) == a ? side : bp, hi = std::min(a, p) == a ? bp : side;
        fe[nf++] = {edge_number(q, lo, hi), (double)bp, 0.5, corner_of(a, side, p, q, bp, 0),
                    corner_of(a, side, p, q, bp, 1)};
      }
      FaceEdge* cr[4];
      int ncr = 0;
      for (int i = 0; i < 4; ++i)
        if (inside(fe[i].c0) != inside(fe[i].c1)) cr[ncr++] = &fe[i];
      if (ncr == 0) continue;
      struct Seg { FaceEdge* a; FaceEdge* b; double ru, rv; } segs[2];
      int ns = 0;
      if (ncr == 2) {
        double ru = 0, rv = 0;
        for (int bp = 0; bp < 2 && !ns; ++bp)
          for (int bq = 0; bq < 2 && !ns; ++bq)
            if (inside(corner_of(a, side, p, q, bp, bq))) { ru = bp; rv = bq; ns = 1; }
        segs[0] = {cr[0], cr[1], ru, rv};
      } else {
        for (int bp = 0; bp < 2; ++bp)
          for (int bq = 0; bq < 2; ++bq) {
            int c = corner_of(a, side, p, q, bp, bq);
            if (!inside(c)) continue;
            FaceEdge* around[2];
            int k = 0;
            for (int i = 0; i < 4; ++i)
              if (cr[i]->c0 == c || cr[i]->c1 == c) around[k++] = cr[i];
            segs[ns++] = {around[0], around[1], (double)bp, (double)bq};
          }
      }
      for (int s = 0; s < ns; ++s) {
        double du = segs[s].b->u - segs[s].a->u, dv = segs[s].b->v - segs[s].a->v;
        double wu = segs[s].ru - segs[s].a->u, wv = segs[s].rv - segs[s].a->v;
        double cr2 = du * wv - dv * wu;
        int from = segs[s].a->id, to = segs[s].b->id;
        if (orient * cr2 > 0) std::swap(from, to);   // keep the inside corner on the right
        next[from] = to;
        crossing[from] = crossing[to] = true;
      }
    }
  }
  bool seen[12] = {};
  int nt = 0;
  for (int e = 0; e < 12; ++e) {
    if (!crossing[e] || seen[e]) continue;
    int loop[12], m = 0;
    int x = e;
    do {
      loop[m++] = x;
      seen[x] = true;
      x = next[x];
    } while (x != e && x >= 0 && m < 12);
    for (int i = 1; i + 1 < m; ++i) {
      tris[(nt * 3) + 0] = (int8_t)loop[0];
      tris[(nt * 3) + 1] = (int8_t)loop[i];
      tris[(nt * 3) + 2] = (int8_t)loop[i + 1];
      ++nt;
    }
  }
  *ntri = (int8_t)nt;
}

__constant__ int8_t c_ntri[256];
__constant__ int8_t c_tris[256 * ISX_MC_MAX_TRI * 3];
// per local edge: axis, start offsets (dx, dy, dz), start corner, end corner
__constant__ int8_t c_edge[12][6];

std::mutex g_table_mu;
bool g_table_done[64] = {};

}  // namespace

void mc_build_table(int8_t* ntri, int8_t* tris) {
  std::memset(tris, -1, 256 * ISX_MC_MAX_TRI * 3);
  for (int c = 0; c < 256; ++c) build_case(c, &ntri[c], &tris[c * ISX_MC_MAX_TRI * 3]);
}

isx_status mc_upload_table(int device) {
  std::lock_guard<std::mutex> lk(g_table_mu);
  if (device < 64 && g_table_done[device]) return ISX_OK;
  int8_t ntri[256], tris[256 * ISX_MC_MAX_TRI * 3];
  mc_build_table(ntri, tris);
  int8_t edge[12][6];
  for (int a = 0; a < 3; ++a) {
    int p = a == 0 ? 1 : 0, q = a == 2 ? 1 : 2;
    for (int t = 0; t < 4; ++t) {
      int off[3] = {0, 0, 0};
      off[p] = t & 1;
      off[q] = t >> 1;
      int c0 = off[0] | (off[1] << 1) | (off[2] << 2);
      int e = 4 * a + t;
      edge[e][0] = (int8_t)a;
      edge[e][1] = (int8_t)off[0];
      edge[e][2] = (int8_t)off[1];
      edge[e][3] = (int8_t)off[2];
      edge[e][4] = (int8_t)c0;
      edge[e][5] = (int8_t)(c0 | (1 << a));
    }
  }
  ISX_CUDA(cudaMemcpyToSymbol(c_ntri, ntri, sizeof(ntri)));
  ISX_CUDA(cudaMemcpyToSymbol(c_tris, tris, sizeof(tris)));
  ISX_CUDA(cudaMemcpyToSymbol(c_edge, edge, sizeof(edge)));
  if (device < 64) g_table_done[device] = true;
  return ISX_OK;
}

// ---- float32 MLP evaluation at points -----------------------------------------------------------
namespace {

constexpr int kEvalPts = 32;

// Points come either as xyz triples or as lattice ids of the (R+1)^3 grid (coordinates
// -1 + 2 i / R, computed directly).
__device__ __forceinline__ void point_xyz(const float* xyz, const uint32_t* ids, int R, int64_t i, float p[3]) {
  if (ids) {
    uint32_t id = ids[i];
    uint32_t n1 = (uint32_t)R + 1u;
    uint32_t ix = id % n1, iy = (id / n1) % n1, iz = id / (n1 * n1);
    float inv = 2.0f / (float)R;
    p[0] = -1.0f + inv * (float)ix;
    p[1] = -1.0f + inv * (float)iy;
    p[2] = -1.0f + inv * (float)iz;
  } else {
    p[0] = xyz[3 * i];
    p[1] = xyz[3 * i + 1];
    p[2] = xyz[3 * i + 2];
  }
}

struct MlpView {
  int n_layers;
  int w;
  int act;                             // isx_activation of the hidden layers
  const float* W0;
  const float* b0;
  const float* Wt[ISX_MAX_LAYERS];
  const float* b[ISX_MAX_LAYERS];
  const float* wout;
  float bout;
};

__global__ void __launch_bounds__(256) k_eval_fp32(MlpView m, const float* xyz, const uint32_t* ids, int R,
                                                   int64_t n, float* out) {
  extern __shared__ float sm[];
  const int w = m.w;
  float* A = sm;                       // [kEvalPts][w]
  float* B = sm + kEvalPts * w;        // [kEvalPts][w]
  __shared__ float pts[kEvalPts][3];
  int64_t p0 = (int64_t)blockIdx.x * kEvalPts;
  if (threadIdx.x < kEvalPts) {
    int64_t i = p0 + threadIdx.x;
    float p[3] = {0.f, 0.f, 0.f};
    if (i < n) point_xyz(xyz, ids, R, i, p);
    pts[threadIdx.x][0] = p[0];
    pts[threadIdx.x][1] = p[1];
    pts[threadIdx.x][2] = p[2];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < kEvalPts * w; idx += blockDim.x) {
    int p = idx / w, nn = idx % w;
    float z = fmaf(m.W0[3 * nn + 2], pts[p][2], fmaf(m.W0[3 * nn + 1], pts[p][1], fmaf(m.W0[3 * nn], pts[p][0], m.b0[nn])));
    A[p * w + nn] = act_fwd(m.act, z);
  }
  __syncthreads();
  for (int l = 1; l < m.n_layers - 1; ++l) {
    const float* Wt = m.Wt[l];
    const float* bb = m.b[l];
    for (int nn = threadIdx.x; nn < w; nn += blockDim.x) {
      float acc[kEvalPts];
#pragma unroll
      for (int p = 0; p < kEvalPts; ++p) acc[p] = bb[nn];
      for (int k = 0; k < w; ++k) {
        float wk = Wt[(size_t)k * w + nn];
#pragma unroll
        for (int p = 0; p < kEvalPts; ++p) acc[p] = fmaf(wk, A[p * w + k], acc[p]);
      }
#pragma unroll
      for (int p = 0; p < kEvalPts; ++p) B[p * w + nn] = act_fwd(m.act, acc[p]);
    }
    __syncthreads();
    float* t = A; A = B; B = t;
  }
  // output layer: one warp per point
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int p = warp; p < kEvalPts; p += blockDim.x >> 5) {
    float s = 0.0f;
    for (int k = lane; k < w; k += 32) s = fmaf(m.wout[k], A[p * w + k], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    int64_t i = p0 + p;
    if (lane == 0 && i < n) out[i] = s + m.bout;
  }
}

}  // namespace

isx_status eval_points_fp32(isx_inr inr, const float* xyz, const uint32_t* lattice_ids, int R, int64_t n,
                            float* out, cudaStream_t st) {
  if (n <= 0) return ISX_OK;
  MlpView m{};
  m.n_layers = inr->n_layers;
  m.w = inr->w;
  m.act = inr->act;
  m.W0 = inr->W[0];
  m.b0 = inr->b[0];
  for (int l = 1; l < inr->n_layers - 1; ++l) {
    m.Wt[l] = inr->Wt[l];
    m.b[l] = inr->b[l];
  }
  m.wout = inr->W[inr->n_layers - 1];
  m.bout = inr->hb[inr->n_layers - 1][0];
  size_t smem = 2ull * kEvalPts * inr->w * sizeof(float);
  static bool attr_set[64] = {};
  if (smem > 48 * 1024 && inr->device < 64 && !attr_set[inr->device]) {
    ISX_CUDA(cudaFuncSetAttribute(k_eval_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set[inr->device] = true;
  }
  int64_t nb = (n + kEvalPts - 1) / kEvalPts;
  {
    prof::Scope _ps(K_EVAL_FP32, st, 2.0 * n * (4.0 * inr->w + (inr->n_layers - 2.0) * inr->w * inr->w), 8.0 * n);
    k_eval_fp32<<<(unsigned)nb, 256, smem, st>>>(m, xyz, lattice_ids, R, n, out);
  }
  ISX_LAUNCH_CHECK("k_eval_fp32");
  return ISX_OK;
}

// ---- corner marking and marching cubes -------------------------------------------------------------
namespace {

__device__ __forceinline__ uint32_t lattice_id(uint32_t i, uint32_t j, uint32_t k, uint32_t n1) {
  return (k * n1 + j) * n1 + i;
}

__global__ void k_mark_corners(const uint32_t* codes, int64_t n, int R, uint8_t* flags) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * 8) return;
  int64_t cell = t >> 3;
  int c = (int)(t & 7);
  uint32_t code = codes[cell];
  uint32_t i = (code & 1023u) + (c & 1), j = ((code >> 10) & 1023u) + ((c >> 1) & 1),
           k = ((code >> 20) & 1023u) + ((c >> 2) & 1);
  flags[lattice_id(i, j, k, (uint32_t)R + 1u)] = 1;
}

// Cells either listed (codes, masks) or implicit (all R^3 cells, every iso-value); corner values
// either through idx_map (compacted points) or directly by lattice id.
struct CellView {
  const uint32_t* codes;
  const uint32_t* masks;
  uint32_t all_mask;
  int R;
  const uint32_t* idx_map;
  const float* values;
};

__device__ __forceinline__ void load_cell(const CellView& v, int64_t cell, uint32_t ijk[3], uint32_t& mask,
                                          float cv[8]) {
  uint32_t code;
  if (v.codes) {
    code = v.codes[cell];
    mask = v.masks[cell];
    ijk[0] = code & 1023u;
    ijk[1] = (code >> 10) & 1023u;
    ijk[2] = (code >> 20) & 1023u;
  } else {
    uint32_t R = (uint32_t)v.R;
    ijk[0] = (uint32_t)(cell % R);
    ijk[1] = (uint32_t)((cell / R) % R);
    ijk[2] = (uint32_t)(cell / ((int64_t)R * R));
    mask = v.all_mask;
  }
  uint32_t n1 = (uint32_t)v.R + 1u;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    uint32_t id = lattice_id(ijk[0] + (c & 1), ijk[1] + ((c >> 1) & 1), ijk[2] + ((c >> 2) & 1), n1);
    cv[c] = v.values[v.idx_map ? v.idx_map[id] : id];
  }
}

__device__ __forceinline__ int cell_case(const float cv[8], float iso) {
  int cs = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) cs |= (cv[c] < iso ? 1 : 0) << c;
  return cs;
}

constexpr int kMcThreads = 256;

// Triangles per cell (counts) and per block (block_tot); with block_ne, also the cells of the block
// that have at least one triangle.
__global__ void __launch_bounds__(kMcThreads) k_mc_count(CellView v, int64_t n, IsoSet iso, int* counts,
                                                         int* block_tot, int* block_ne) {
  int64_t cell = blockIdx.x * (int64_t)kMcThreads + threadIdx.x;
  int cnt = 0;
  if (cell < n) {
    uint32_t ijk[3], mask;
    float cv[8];
    load_cell(v, cell, ijk, mask, cv);
    for (int q = 0; q < iso.n; ++q)
      if ((mask >> q) & 1u) cnt += c_ntri[cell_case(cv, iso.c[q])];
    counts[cell] = cnt;
  }
  __shared__ int red[2][kMcThreads / 32];
  int s = cnt, e = cnt > 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    e += __shfl_xor_sync(0xffffffffu, e, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s;
    red[1][threadIdx.x >> 5] = e;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0, te = 0;
    for (int q = 0; q < kMcThreads / 32; ++q) {
      t += red[0][q];
      te += red[1][q];
    }
    block_tot[blockIdx.x] = t;
    if (block_ne) block_ne[blockIdx.x] = te;
  }
}

// Exclusive scan of v over the block (kMcThreads threads); `wsum` holds kMcThreads / 32 ints.
__device__ __forceinline__ int block_excl_scan_int(int v, int* wsum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int s = lane < kMcThreads / 32 ? wsum[lane] : 0;
    int si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += t;
    }
    if (lane < kMcThreads / 32) wsum[lane] = si - s;
  }
  __syncthreads();
  return wsum[warp] + incl - v;
}

// The cells with at least one triangle, in cell order, with the mask of the isos they have
// triangles for (dense extraction's list of truly crossing cells).  ne_off: per-block offsets.
struct NonemptyOut {
  const int64_t* ne_off = nullptr;
  uint32_t* code = nullptr;
  uint32_t* mask = nullptr;
  int64_t cap = 0;
};

__global__ void __launch_bounds__(kMcThreads) k_mc_emit(CellView v, int64_t n, IsoSet iso, const int* counts,
                                                        const int64_t* block_off, float* tri_vert,
                                                        int64_t* tri_edge, int32_t* tri_iso, uint32_t* tri_cell,
                                                        NonemptyOut ne) {
  int64_t cell = blockIdx.x * (int64_t)kMcThreads + threadIdx.x;
  int cnt = cell < n ? counts[cell] : 0;
  __shared__ int wsum[kMcThreads / 32];
  const int ex = block_excl_scan_int(cnt, wsum);          // block exclusive scan of cnt
  int ex_ne = 0;
  if (ne.ne_off) {
    __syncthreads();
    ex_ne = block_excl_scan_int(cnt > 0 ? 1 : 0, wsum);   // ... and of the non-empty flags
  }
  if (cell >= n || cnt == 0) return;
  int64_t off = block_off[blockIdx.x] + ex;
  uint32_t ijk[3], mask;
  float cv[8];
  load_cell(v, cell, ijk, mask, cv);
  if (ne.ne_off) {
    const int64_t a = ne.ne_off[blockIdx.x] + ex_ne;
    if (ne.code && a < ne.cap) {
      uint32_t m = 0;
      for (int q = 0; q < iso.n; ++q)
        if (((mask >> q) & 1u) && c_ntri[cell_case(cv, iso.c[q])] > 0) m |= 1u << q;
      ne.code[a] = ijk[0] | (ijk[1] << 10) | (ijk[2] << 20);
      ne.mask[a] = m;
    }
  }
  uint32_t n1 = (uint32_t)v.R + 1u;
  float inv = 2.0f / (float)v.R;
  for (int q = 0; q < iso.n; ++q) {
    if (!((mask >> q) & 1u)) continue;
    float c = iso.c[q];
    int cs = cell_case(cv, c);
    int nt = c_ntri[cs];
    for (int t = 0; t < nt; ++t) {
      for (int e3 = 0; e3 < 3; ++e3) {
        int e = c_tris[(cs * ISX_MC_MAX_TRI + t) * 3 + e3];
        int a = c_edge[e][0];
        uint32_t pi = ijk[0] + c_edge[e][1], pj = ijk[1] + c_edge[e][2], pk = ijk[2] + c_edge[e][3];
        float va = cv[c_edge[e][4]], vb = cv[c_edge[e][5]];
        float tt = (c - va) / (vb - va);      // from the endpoint with the lower lattice index
        float x = -1.0f + inv * (float)pi, y = -1.0f + inv * (float)pj, z = -1.0f + inv * (float)pk;
        if (a == 0) x += inv * tt;
        else if (a == 1) y += inv * tt;
        else z += inv * tt;
        float* vo = tri_vert + (off * 3 + e3) * 3;
        vo[0] = x;
        vo[1] = y;
        vo[2] = z;
        tri_edge[off * 3 + e3] = 3 * (int64_t)lattice_id(pi, pj, pk, n1) + a;
      }
      tri_iso[off] = q;
      if (tri_cell) tri_cell[off] = ijk[0] | (ijk[1] << 10) | (ijk[2] << 20);
      ++off;
    }
  }
}

}  // namespace

isx_status mark_corners(const uint32_t* codes, int64_t n, int R, uint8_t* flags, cudaStream_t st) {
  if (n == 0) return ISX_OK;
  int64_t tot = n * 8;
  {
    prof::Scope _ps(K_MARK, st, 0, 0);
    k_mark_corners<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(codes, n, R, flags);
  }
  ISX_LAUNCH_CHECK("k_mark_corners");
  return ISX_OK;
}

// Marching cubes over n cells; if tri capacity suffices emits, else only reports the count.
isx_status marching_cubes(isx_inr inr, const uint32_t* codes, const uint32_t* masks, int64_t n, int R,
                          const uint32_t* idx_map, const float* values, const IsoSet& iso, isx_mesh* mesh,
                          bool count_nonempty, cudaStream_t st) {
  mesh->n_tris = 0;
  if (n == 0) return ISX_OK;
  ISX_TRY(mc_upload_table(inr->device));
  CellView v{codes, masks, (iso.n >= 32) ? 0xffffffffu : ((1u << iso.n) - 1u), R, idx_map, values};
  int64_t nb = (n + kMcThreads - 1) / kMcThreads;
  auto& ws = inr->ws;
  ISX_TRY(ws[WS_TRI_COUNT].ensure((size_t)n * sizeof(int), "tri counts"));
  size_t head = ((nb * sizeof(int) + 15) / 16) * 16;
  // [block triangle totals][block non-empty totals][triangle offsets][non-empty offsets][2 totals]
  ISX_TRY(ws[WS_TRI_OFFSET].ensure(2 * head + 2 * nb * sizeof(int64_t) + 16 * sizeof(int64_t), "tri offsets"));
  int* counts = ws[WS_TRI_COUNT].as<int>();
  int* btot = ws[WS_TRI_OFFSET].as<int>();
  int* bne = reinterpret_cast<int*>(ws[WS_TRI_OFFSET].as<char>() + head);
  int64_t* boff = reinterpret_cast<int64_t*>(ws[WS_TRI_OFFSET].as<char>() + 2 * head);
  int64_t* neoff = boff + nb;
  int64_t* d_total = neoff + nb;
  int64_t* d_ne_total = d_total + 2;
  {
    prof::Scope _ps(K_MC_COUNT, st, 0, 0);
    k_mc_count<<<(unsigned)nb, kMcThreads, 0, st>>>(v, n, iso, counts, btot, count_nonempty ? bne : nullptr);
  }
  ISX_LAUNCH_CHECK("k_mc_count");
  ISX_TRY(scan_block_counts(inr, btot, nb, boff, d_total, st));
  if (count_nonempty) ISX_TRY(scan_block_counts(inr, bne, nb, neoff, d_ne_total, st));
  int64_t totals[3] = {0, 0, 0};
  ISX_CUDA(cudaMemcpyAsync(totals, d_total, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  ISX_CUDA(cudaStreamSynchronize(st));
  const int64_t total = totals[0];
  mesh->n_tris = total;
  if (count_nonempty) mesh->n_active = totals[2];
  if (total > mesh->tri_cap) {
    set_error("triangle capacity exceeded");
    return ISX_ERR_CAPACITY;
  }
  if (total == 0) return ISX_OK;
  if (!mesh->d_tri_vert || !mesh->d_tri_edge || !mesh->d_tri_iso) {
    set_error("null triangle output buffer");
    return ISX_ERR_ARG;
  }
  NonemptyOut ne;
  if (count_nonempty) {
    ne.ne_off = neoff;
    if (mesh->d_active_code && mesh->d_active_mask && totals[2] <= mesh->active_cap) {
      ne.code = mesh->d_active_code;
      ne.mask = mesh->d_active_mask;
      ne.cap = mesh->active_cap;
    }
  }
  {
    prof::Scope _ps(K_MC_EMIT, st, 0, 0);
    k_mc_emit<<<(unsigned)nb, kMcThreads, 0, st>>>(v, n, iso, counts, boff, mesh->d_tri_vert, mesh->d_tri_edge,
                                                   mesh->d_tri_iso, mesh->d_tri_cell, ne);
  }
  ISX_LAUNCH_CHECK("k_mc_emit");
  return ISX_OK;
}

}  // namespace isx
