// S-NFC neighbour search (Sec. II-B, Eq. neardef) and the numbering of unknowns (Sec. II-A).
//
// Wires are binned into a uniform grid of cell side h >= r_c and renumbered by (cell, caller
// index); a wire's S-NFC partners then lie in the 27 surrounding cells, whose wires occupy nine
// contiguous index ranges.  One warp per wire tests 32 candidates at a time in float64 and
// compacts the kept ones with a ballot, so each block-row comes out sorted by column.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "ctx.h"

namespace swm {

namespace {

constexpr int64_t kMaxCells = int64_t(1) << 24;

struct Grid {
  double x0, y0, z0, h;
  int nx, ny, nz;
};

__device__ __forceinline__ int cell_coord(double v, double v0, double h, int n) {
  int i = (int)floor((v - v0) / h);
  return min(max(i, 0), n - 1);
}

__global__ void k_cell_ids(const double* __restrict__ c, int64_t nw, Grid g, int32_t* __restrict__ cid,
                           int32_t* __restrict__ cnt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nw) return;
  const int ix = cell_coord(c[3 * i], g.x0, g.h, g.nx);
  const int iy = cell_coord(c[3 * i + 1], g.y0, g.h, g.ny);
  const int iz = cell_coord(c[3 * i + 2], g.z0, g.h, g.nz);
  const int id = (iz * g.ny + iy) * g.nx + ix;
  cid[i] = id;
  atomicAdd(&cnt[id], 1);
}

// Each wire into a free slot of its cell's range (the cell count, counted down, numbers the slots).
__global__ void k_scatter_unordered(const int32_t* __restrict__ cid, int64_t nw, const int64_t* __restrict__ cstart,
                                    int32_t* __restrict__ cnt, int32_t* __restrict__ tmp) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nw) return;
  const int id = cid[i];
  const int64_t pos = cstart[id] + atomicSub(&cnt[id], 1) - 1;
  tmp[pos] = (int32_t)i;
}

// Deterministic order inside a cell: a wire's rank is the number of wires of its cell with a
// smaller caller index.  Wire i goes to position s + rank: the permutation, its inverse, the sorted
// cell ids, and the wire's geometry written in internal order (m = segments - 1 unknowns).
__global__ void k_rank_and_place(const int32_t* __restrict__ cid, int64_t nw, const int64_t* __restrict__ cstart,
                                 const int32_t* __restrict__ tmp, int32_t* __restrict__ perm,
                                 int32_t* __restrict__ iperm, int32_t* __restrict__ cid_sorted,
                                 const double* __restrict__ uc, const double* __restrict__ ut,
                                 const double* __restrict__ uL, const double* __restrict__ ua,
                                 const int32_t* __restrict__ uns, double* cx, double* cy, double* cz, double* tx,
                                 double* ty, double* tz, double* L, double* a, int32_t* ns, int32_t* m) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nw) return;
  const int id = cid[i];
  const int64_t s = cstart[id], e = cstart[id + 1];
  int64_t r = 0;
  for (int64_t t = s; t < e; ++t) r += (tmp[t] < (int32_t)i);
  const int64_t p = s + r;
  perm[p] = (int32_t)i;
  iperm[i] = (int32_t)p;
  cid_sorted[p] = id;
  cx[p] = uc[3 * i];
  cy[p] = uc[3 * i + 1];
  cz[p] = uc[3 * i + 2];
  tx[p] = ut[3 * i];
  ty[p] = ut[3 * i + 1];
  tz[p] = ut[3 * i + 2];
  L[p] = uL[i];
  a[p] = ua[i];
  ns[p] = uns[i];
  m[p] = uns[i] - 1;
}

__global__ void k_user_m(int64_t nw, const int32_t* __restrict__ uns, int32_t* __restrict__ um) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < nw) um[i] = uns[i] - 1;
}

__global__ void k_uoff_by_internal(int64_t nw, const int32_t* __restrict__ perm, const int64_t* __restrict__ uoff_user,
                                   int64_t* __restrict__ uoff) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < nw) uoff[p] = uoff_user[perm[p]];
}

// Per-row sizes gathered by the counting pass of k_pairs: kept blocks, kept blocks above the
// diagonal, and the row lengths and entry counts of both layouts (with and without the diagonal
// block), so that one read-back after one scan sizes every pattern array.
struct RowCounts {
  int32_t* cnt;    // kept partners
  int64_t* ucnt;   // partners q > p
  int32_t* K_f;    // sum of m_q over kept q
  int32_t* K_o;    // the same without q = p
  int64_t* ent_f;  // m_p K_f
  int64_t* ent_o;  // m_p K_o
  int64_t* msq;    // m_p^2
};

// mode 0: count kept partners per wire (and the sizes in RowCounts); mode 1: write them (sorted)
// into col, with the position of each row's diagonal block and every block's first column in the
// full layout and in the layout without the diagonal block (-1 for the diagonal).  One warp per wire: lanes 0..8 look up the nine (z, y) rows of three cells around the
// wire's cell at once (each a contiguous range of the renumbered wires), a warp scan lays the
// ranges end to end, and the warp tests 32 candidates per pass, so a wire costs about three
// dependent memory round trips whatever its cell occupancy.  Candidates are visited in increasing
// index order (rows in cell order), so the ballot compaction writes each row's partners sorted.
__global__ void k_pairs(int64_t nw, const double* __restrict__ cx, const double* __restrict__ cy,
                        const double* __restrict__ cz, const int32_t* __restrict__ cid, const int64_t* __restrict__ cstart,
                        Grid g, double rc2, int dense, int mode, RowCounts rc, const int32_t* __restrict__ m,
                        const int64_t* __restrict__ row_ptr, int32_t* __restrict__ col, int64_t* __restrict__ diag_b,
                        int32_t* __restrict__ colpos_f, int32_t* __restrict__ colpos_o) {
  const int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (p >= nw) return;
  const int id = cid[p];
  const int ix = id % g.nx, iy = (id / g.nx) % g.ny, iz = id / (g.nx * g.ny);
  // this lane's row range (lanes 0..8)
  int64_t q0 = 0, len = 0;
  if (lane < 9) {
    const int z = iz + lane / 3 - 1, y = iy + lane % 3 - 1;
    if (z >= 0 && z < g.nz && y >= 0 && y < g.ny) {
      const int x0 = max(ix - 1, 0), x1 = min(ix + 1, g.nx - 1);
      const int64_t c0 = ((int64_t)z * g.ny + y) * g.nx + x0;
      const int64_t c1 = ((int64_t)z * g.ny + y) * g.nx + x1;
      q0 = cstart[c0];
      len = cstart[c1 + 1] - q0;
    }
  }
  const double px = cx[p], py = cy[p], pz = cz[p];
  int64_t incl = len;
#pragma unroll
  for (int o = 1; o < 16; o <<= 1) {
    const int64_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int64_t total = __shfl_sync(0xffffffffu, incl, 8);
  // every lane keeps the nine ranges' starts in the flat order and their first indices
  int64_t fs[9], qs[9];
#pragma unroll
  for (int r = 0; r < 9; ++r) {
    const int64_t e = __shfl_sync(0xffffffffu, incl - len, r);
    fs[r] = e;
    qs[r] = __shfl_sync(0xffffffffu, q0, r) - e;  // q = f + qs[r] inside range r
  }
  int64_t count = 0;
  int32_t msum = 0, nup = 0;  // this lane's kept m_q and kept q > p (counting pass)
  const int64_t base = mode ? row_ptr[p] : 0;
  // writing pass: running offsets of the kept blocks' columns in the full layout and in the layout
  // without the diagonal block (whose m_p columns the second one skips)
  int32_t kf = 0, mp_seen = 0;
  const int32_t mp_w = mode ? m[p] : 0;
  for (int64_t fb = 0; fb < total; fb += 32) {
    const int64_t f = fb + lane;
    bool keep = false;
    int64_t q = 0;
    if (f < total) {
      int64_t off = qs[0];
#pragma unroll
      for (int r = 1; r < 9; ++r)
        if (f >= fs[r]) off = qs[r];  // empty ranges share their start with the next one
      q = f + off;
      if (dense) {
        keep = true;
      } else {
        const double dx = px - cx[q], dyy = py - cy[q], dzz = pz - cz[q];
        // (dx*dx + dy*dy) + dz*dz, each operation rounded separately (no contraction)
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dyy, dyy)), __dmul_rn(dzz, dzz));
        keep = d2 <= rc2;
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (mode) {
      // column positions: exclusive warp scan of m_q over the kept lanes (in q order)
      const int32_t mq = keep ? m[q] : 0;
      int32_t incl = mq;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const unsigned dmask = __ballot_sync(0xffffffffu, keep && q == p);
      if (keep) {
        const int64_t b = base + count + __popc(bal & ((1u << lane) - 1u));
        col[b] = (int32_t)q;
        const int32_t pf = kf + incl - mq;
        colpos_f[b] = pf;
        const bool diag_before = mp_seen || (dmask & ((1u << lane) - 1u));
        colpos_o[b] = q == p ? -1 : pf - (diag_before ? mp_w : 0);
        if (q == p) diag_b[p] = b;
      }
      kf += __shfl_sync(0xffffffffu, incl, 31);
      if (dmask) mp_seen = 1;
    }
    if (!mode && keep) {
      msum += m[q];
      nup += q > p ? 1 : 0;
    }
    count += __popc(bal);
  }
  if (!mode) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      msum += __shfl_xor_sync(0xffffffffu, msum, o);
      nup += __shfl_xor_sync(0xffffffffu, nup, o);
    }
    if (lane == 0) {
      const int32_t mp = m[p];
      rc.cnt[p] = (int32_t)count;
      rc.ucnt[p] = nup;
      rc.K_f[p] = msum;
      rc.K_o[p] = msum - mp;  // the diagonal block (distance 0) is always kept
      rc.ent_f[p] = (int64_t)mp * msum;
      rc.ent_o[p] = (int64_t)mp * (msum - mp);
      rc.msq[p] = (int64_t)mp * mp;
    }
  }
}

__device__ __forceinline__ int64_t find_in_row(const int32_t* __restrict__ col, int64_t b, int64_t e, int32_t key) {
  while (b < e) {
    const int64_t mid = (b + e) >> 1;
    if (col[mid] < key)
      b = mid + 1;
    else
      e = mid;
  }
  return b;
}

__global__ void k_transpose_and_upper(int64_t nw, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                      const int64_t* __restrict__ diag_b, const int64_t* __restrict__ ubase,
                                      int64_t* __restrict__ bt, int64_t* __restrict__ ublk) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nw) return;
  const int64_t b0 = row_ptr[p], b1 = row_ptr[p + 1];
  for (int64_t b = b0; b < b1; ++b) {
    const int32_t q = col[b];
    bt[b] = find_in_row(col, row_ptr[q], row_ptr[q + 1], (int32_t)p);
  }
  int64_t u = ubase[p];
  for (int64_t b = diag_b[p] + 1; b < b1; ++b) ublk[u++] = b;
}

// Column maps of both layouts (with and without the diagonal blocks), one thread per block-row.
// Column maps of both layouts, and for the Krylov kernels each scalar row's wire and its 16-byte
// descriptor in the off-diagonal layout (first value, first column-map entry, length).
__global__ void k_colmap(int64_t nw, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                         const int32_t* __restrict__ m, const int64_t* __restrict__ off, Layout a, Layout b2,
                         int32_t* __restrict__ rowwire, RowInfo* __restrict__ rinfo) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nw) return;
  {
    const int K = b2.K[p];
    const int64_t o0 = off[p], o1 = off[p + 1];
    for (int64_t n = o0; n < o1; ++n) {
      rowwire[n] = (int32_t)p;
      rinfo[n] = RowInfo{b2.rowbase[p] + (n - o0) * K, (int32_t)b2.cmbase[p], K};
    }
  }
  for (int64_t b = row_ptr[p]; b < row_ptr[p + 1]; ++b) {
    const int32_t q = col[b];
    const int32_t ca = a.colpos[b], cb = b2.colpos[b];
    for (int j = 0; j < m[q]; ++j) {
      const int32_t v = (int32_t)(off[q] + j);
      if (ca >= 0) a.colmap[a.cmbase[p] + ca + j] = v;
      if (cb >= 0) b2.colmap[b2.cmbase[p] + cb + j] = v;
    }
  }
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, ceil_div(n, t)); }

int alloc_layout(swm_ctx* ctx, Layout& lay, int32_t* K, int32_t* colpos) {
  lay.K = K;
  lay.colpos = colpos;
  SWM_TRY(dalloc(ctx, ctx->pattern_bufs, (void**)&lay.rowbase, sizeof(int64_t) * (ctx->nw + 1)));
  SWM_TRY(dalloc(ctx, ctx->pattern_bufs, (void**)&lay.cmbase, sizeof(int64_t) * (ctx->nw + 1)));
  return SWM_OK;
}

}  // namespace

int ensure_user_offsets(swm_ctx* ctx) {
  if (ctx->uoff) return SWM_OK;
  const int64_t nw = ctx->nw;
  std::vector<Buf> tmp;
  int32_t* um = nullptr;
  SWM_TRY(dalloc(ctx, tmp, (void**)&um, sizeof(int32_t) * nw));
  k_user_m<<<nblk(nw, 256), 256, 0, ctx->stream>>>(nw, ctx->u_ns, um);
  SWM_LAUNCHED();
  SWM_TRY(dalloc(ctx, ctx->pattern_bufs, (void**)&ctx->uoff_user, sizeof(int64_t) * (nw + 1)));
  SWM_TRY(exclusive_scan_i32_to_i64(ctx, um, ctx->uoff_user, nw, nullptr));
  SWM_TRY(dalloc(ctx, ctx->pattern_bufs, (void**)&ctx->uoff, sizeof(int64_t) * nw));
  k_uoff_by_internal<<<nblk(nw, 256), 256, 0, ctx->stream>>>(nw, ctx->perm, ctx->uoff_user, ctx->uoff);
  SWM_LAUNCHED();
  dfree_group(ctx, tmp);
  return SWM_OK;
}

int build_pattern(swm_ctx* ctx) {
  const int64_t nw = ctx->nw;
  cudaStream_t st = ctx->stream;
  std::vector<Buf> tmp;
  auto& B = ctx->pattern_bufs;

  // --- bounding box of the centres (computed when the cloud was loaded)
  const double* hb = ctx->bbox;

  // --- grid (cell side slightly above r_c so a pair at exactly r_c is never two cells apart)
  Grid g;
  g.x0 = hb[0];
  g.y0 = hb[1];
  g.z0 = hb[2];
  const double ext = std::max({hb[3] - hb[0], hb[4] - hb[1], hb[5] - hb[2], 0.0});
  if (ctx->dense) {
    g.h = ext * 2.0 + 1.0;
  } else {
    g.h = ctx->rc * (1.0 + 1e-9) + 1e-300;
  }
  auto dims = [&](double h, int64_t& nx, int64_t& ny, int64_t& nz) {
    nx = (int64_t)std::floor((hb[3] - hb[0]) / h) + 1;
    ny = (int64_t)std::floor((hb[4] - hb[1]) / h) + 1;
    nz = (int64_t)std::floor((hb[5] - hb[2]) / h) + 1;
  };
  int64_t nx, ny, nz;
  dims(g.h, nx, ny, nz);
  // at most 64 cells per wire (larger cells only add candidates to the distance test, more cells
  // only add empty ones to scan)
  const double max_cells = std::min<double>((double)kMaxCells, std::max<double>(4096.0, 64.0 * (double)nw));
  while ((double)nx * (double)ny * (double)nz > max_cells) {
    g.h *= 1.05 * std::cbrt((double)nx * ny * nz / max_cells);
    dims(g.h, nx, ny, nz);
  }
  g.nx = (int)nx;
  g.ny = (int)ny;
  g.nz = (int)nz;
  const int64_t ncell = nx * ny * nz;

  // --- bin and renumber by (cell, caller index)
  int32_t *cid = nullptr, *cnt = nullptr, *tmpidx = nullptr, *cid_s = nullptr;
  int64_t* cstart = nullptr;
  SWM_TRY(dalloc(ctx, tmp, (void**)&cid, sizeof(int32_t) * nw));
  SWM_TRY(dalloc(ctx, tmp, (void**)&cnt, sizeof(int32_t) * ncell));
  SWM_TRY(dalloc(ctx, tmp, (void**)&tmpidx, sizeof(int32_t) * nw));
  SWM_TRY(dalloc(ctx, tmp, (void**)&cid_s, sizeof(int32_t) * nw));
  SWM_TRY(dalloc(ctx, tmp, (void**)&cstart, sizeof(int64_t) * (ncell + 1)));
  SWM_CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ncell, st));
  k_cell_ids<<<nblk(nw, 256), 256, 0, st>>>(ctx->u_c, nw, g, cid, cnt);
  SWM_LAUNCHED();
  SWM_TRY(exclusive_scan_i32_to_i64(ctx, cnt, cstart, ncell, nullptr));
  k_scatter_unordered<<<nblk(nw, 256), 256, 0, st>>>(cid, nw, cstart, cnt, tmpidx);
  SWM_LAUNCHED();
  SWM_TRY(dalloc(ctx, B, (void**)&ctx->perm, sizeof(int32_t) * nw));
  SWM_TRY(dalloc(ctx, B, (void**)&ctx->iperm, sizeof(int32_t) * nw));

  // --- order inside cells, geometry in internal order, numbering of unknowns (a0)
  double** geo[8] = {&ctx->cx, &ctx->cy, &ctx->cz, &ctx->tx, &ctx->ty, &ctx->tz, &ctx->L, &ctx->a};
  for (auto pp : geo) SWM_TRY(dalloc(ctx, B, (void**)pp, sizeof(double) * nw));
  int32_t* m = nullptr;
  SWM_TRY(dalloc(ctx, B, (void**)&ctx->ns, sizeof(int32_t) * nw));
  SWM_TRY(dalloc(ctx, B, (void**)&m, sizeof(int32_t) * nw));
  k_rank_and_place<<<nblk(nw, 256), 256, 0, st>>>(cid, nw, cstart, tmpidx, ctx->perm, ctx->iperm, cid_s, ctx->u_c,
                                                  ctx->u_t, ctx->u_L, ctx->u_a, ctx->u_ns, ctx->cx, ctx->cy, ctx->cz,
                                                  ctx->tx, ctx->ty, ctx->tz, ctx->L, ctx->a, ctx->ns, m);
  SWM_LAUNCHED();
  SWM_TRY(dalloc(ctx, B, (void**)&ctx->off, sizeof(int64_t) * (nw + 1)));  // scanned with the row counts below
  ctx->uoff = nullptr;  // caller-order offsets are made on first use (ensure_user_offsets)
  ctx->uoff_user = nullptr;

  // --- S-NFC pairs (a1): count (with the per-row sizes), one merged scan, one read-back, write
  int64_t *ucnt = nullptr, *ubase = nullptr, *ent_f = nullptr, *ent_o = nullptr, *msq = nullptr;
  int32_t *rcnt = nullptr, *Kf = nullptr, *Ko = nullptr, *cpf = nullptr, *cpo = nullptr;
  SWM_TRY(dalloc(ctx, tmp, (void**)&rcnt, sizeof(int32_t) * nw));
  SWM_TRY(dalloc(ctx, tmp, (void**)&ucnt, sizeof(int64_t) * nw));
  SWM_TRY(dalloc(ctx, tmp, (void**)&ubase, sizeof(int64_t) * (nw + 1)));
  SWM_TRY(dalloc(ctx, tmp, (void**)&ent_f, sizeof(int64_t) * nw));
  SWM_TRY(dalloc(ctx, tmp, (void**)&ent_o, sizeof(int64_t) * nw));
  SWM_TRY(dalloc(ctx, tmp, (void**)&msq, sizeof(int64_t) * nw));
  SWM_TRY(dalloc(ctx, B, (void**)&Kf, sizeof(int32_t) * nw));
  SWM_TRY(dalloc(ctx, B, (void**)&Ko, sizeof(int32_t) * nw));
  SWM_TRY(dalloc(ctx, B, (void**)&ctx->row_ptr, sizeof(int64_t) * (nw + 1)));
  SWM_TRY(dalloc(ctx, B, (void**)&ctx->diag_b, sizeof(int64_t) * nw));
  SWM_TRY(alloc_layout(ctx, ctx->full, Kf, nullptr));
  SWM_TRY(alloc_layout(ctx, ctx->offd, Ko, nullptr));
  SWM_TRY(dalloc(ctx, B, (void**)&ctx->minv_off, sizeof(int64_t) * (nw + 1)));
  const double rc2 = ctx->dense ? 0.0 : ctx->rc * ctx->rc;
  RowCounts rcs{rcnt, ucnt, Kf, Ko, ent_f, ent_o, msq};
  ctx->prof_begin(SWM_K_PAIRS);
  k_pairs<<<nblk(nw * 32, 256), 256, 0, st>>>(nw, ctx->cx, ctx->cy, ctx->cz, cid_s, cstart, g, rc2,
                                              ctx->dense ? 1 : 0, 0, rcs, m, nullptr, nullptr, nullptr, nullptr,
                                              nullptr);
  ctx->prof_end(SWM_K_PAIRS);
  SWM_LAUNCHED();
  {
    const void* in[8] = {m, rcnt, ucnt, ent_f, Kf, ent_o, Ko, msq};
    const int is64[8] = {0, 0, 1, 1, 0, 1, 0, 1};
    int64_t* out[8] = {ctx->off, ctx->row_ptr, ubase, ctx->full.rowbase, ctx->full.cmbase, ctx->offd.rowbase,
                       ctx->offd.cmbase, ctx->minv_off};
    // the totals side by side, read back with one copy to pinned memory
    int64_t* tot = nullptr;
    SWM_TRY(dalloc(ctx, tmp, (void**)&tot, sizeof(int64_t) * 8));
    SWM_TRY(exclusive_scan_multi(ctx, 8, in, is64, out, nw, tot));
    SWM_TRY(ensure_poll_slots(ctx));
    int64_t* h = reinterpret_cast<int64_t*>(static_cast<char*>(ctx->pinned_state) + kIngestSlotOffset);
    SWM_CK(cudaMemcpyAsync(h, tot, sizeof(int64_t) * 8, cudaMemcpyDeviceToHost, st));
    SWM_CK(cudaStreamSynchronize(st));
    const int64_t v[7] = {h[0], h[1], h[3], h[4], h[5], h[6], h[7]};  // totals[2] (upper blocks) unused
    ctx->N = v[0];
    ctx->nb = v[1];
    ctx->full.nval = v[2];
    ctx->full.ncm = v[3];
    ctx->offd.nval = v[4];
    ctx->offd.ncm = v[5];
    ctx->nminv = v[6];
  }
  if (ctx->nb > INT32_MAX / 2) return ctx->fail(SWM_EINVAL, "too many kept blocks for 32-bit positions");
  SWM_TRY(dalloc(ctx, B, (void**)&ctx->col, sizeof(int32_t) * ctx->nb));
  SWM_TRY(dalloc(ctx, B, (void**)&cpf, sizeof(int32_t) * ctx->nb));
  SWM_TRY(dalloc(ctx, B, (void**)&cpo, sizeof(int32_t) * ctx->nb));
  ctx->full.colpos = cpf;
  ctx->offd.colpos = cpo;
  ctx->prof_begin(SWM_K_PAIRS);
  k_pairs<<<nblk(nw * 32, 256), 256, 0, st>>>(nw, ctx->cx, ctx->cy, ctx->cz, cid_s, cstart, g, rc2,
                                              ctx->dense ? 1 : 0, 1, rcs, m, ctx->row_ptr, ctx->col, ctx->diag_b,
                                              cpf, cpo);
  ctx->prof_end(SWM_K_PAIRS);
  SWM_LAUNCHED();

  // --- the transpose map with the upper-triangle block list, and the column maps on the build's
  // second stream when it exists (both need the diagonal blocks and column positions that the
  // writing pass of k_pairs produced)
  // the S-NFC pattern is symmetric, so the blocks above the diagonal are half the off-diagonal ones
  ctx->nup = (ctx->nb - nw) / 2;
  SWM_TRY(dalloc(ctx, B, (void**)&ctx->bt, sizeof(int64_t) * ctx->nb));
  SWM_TRY(dalloc(ctx, B, (void**)&ctx->ublk, sizeof(int64_t) * std::max<int64_t>(1, ctx->nup)));
  SWM_TRY(dalloc(ctx, B, (void**)&ctx->full.colmap, sizeof(int32_t) * std::max<int64_t>(1, ctx->full.ncm)));
  SWM_TRY(dalloc(ctx, B, (void**)&ctx->offd.colmap, sizeof(int32_t) * std::max<int64_t>(1, ctx->offd.ncm)));
  if (ctx->offd.ncm > INT32_MAX) return ctx->fail(SWM_EINVAL, "column map too large for 32-bit offsets");
  SWM_TRY(dalloc(ctx, B, (void**)&ctx->rowwire, sizeof(int32_t) * std::max<int64_t>(1, ctx->N)));
  SWM_TRY(dalloc(ctx, B, &ctx->rowinfo, sizeof(RowInfo) * std::max<int64_t>(1, ctx->N)));
  cudaStream_t s2 = ctx->side ? ctx->side : st;
  if (ctx->side) {
    SWM_CK(cudaEventRecord(ctx->side_ev[0], st));
    SWM_CK(cudaStreamWaitEvent(s2, ctx->side_ev[0], 0));
  }
  // column maps (positions from the writing pass, offsets, multiplicities) and the row descriptors
  k_colmap<<<nblk(nw, 256), 256, 0, s2>>>(nw, ctx->row_ptr, ctx->col, m, ctx->off, ctx->full, ctx->offd,
                                          ctx->rowwire, (RowInfo*)ctx->rowinfo);
  SWM_LAUNCHED();
  k_transpose_and_upper<<<nblk(nw, 256), 256, 0, st>>>(nw, ctx->row_ptr, ctx->col, ctx->diag_b, ubase, ctx->bt,
                                                       ctx->ublk);
  SWM_LAUNCHED();
  if (ctx->side) {
    SWM_CK(cudaEventRecord(ctx->side_ev[1], s2));
    SWM_CK(cudaStreamWaitEvent(st, ctx->side_ev[1], 0));
  }
  ctx->m = m;
  dfree_group(ctx, tmp);
  return SWM_OK;
}

}  // namespace swm
