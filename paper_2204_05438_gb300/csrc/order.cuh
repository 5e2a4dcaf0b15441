// Ordering of the pieces of one split polygon (Section 3.2.3's recursion),
// shared by the per-polygon kernel (k_poly_order) and the block that repairs a long
// polygon (k_long_repair).
//
// The processed split edges are non-crossing chords of the polygon's disk, so
// chords and pieces form a tree.  The recursion cuts the chord of the smallest tip
// first and emits the tip->x side before the other; the same order comes from
// merging pieces across chords in decreasing tip order (union-find), each merge
// making a node whose left child holds the tip->x side, and reading the leaves in
// order.  Scratch: 24 ints per tip of the polygon.
#pragma once

#include "walk.cuh"

namespace polylla {

__device__ __forceinline__ void heap_sift(int* key, int* val, int root, int n) {
  for (;;) {
    int c = 2 * root + 1;
    if (c >= n) return;
    if (c + 1 < n && key[c + 1] > key[c]) ++c;
    if (key[root] >= key[c]) return;
    int t = key[root]; key[root] = key[c]; key[c] = t;
    t = val[root]; val[root] = val[c]; val[c] = t;
    root = c;
  }
}

__device__ __forceinline__ void order_pieces(const DevMesh& M, PolyArrays P, TipArrays T, FinalPieces F, Counters* C,
                             long long i, int* scratch, int src) {
  const int nt = P.ntip[i];
  const long long tb = P.tipbase[i];
  const int W = 2 * nt + 1;
  int* chord_k = scratch;              // processed chords (tip entries), then sorted
  int* chord_b = chord_k + nt;         // their tip vertices (sort keys)
  int* nodeof = chord_b + nt;          // record offset (q - 2 tb) -> piece node
  int* node_rec = nodeof + 2 * nt;     // piece node -> its naming record
  int* uf = node_rec + W;
  int* left = uf + W;
  int* right = left + W;
  int* cnt = right + W;
  int* pos = cnt + W;  // component -> tree node while merging, then in-order start
  // 1. processed chords and piece nodes (a piece's node is its naming record)
  int ns = 0, npieces = 0;
  for (int j = 0; j < nt; ++j) {
    const long long k = tb + j;
    if (T.state[k] != 1 || T.o[k] < 0) continue;
    chord_k[ns] = (int)k;
    chord_b[ns] = M.tri[T.o[k]];
    ++ns;
  }
  bool bad = (ns == 0);
  for (int c = 0; c < ns && !bad; ++c) {
    for (int side = 0; side < 2; ++side) {
      const long long q = 2ll * chord_k[c] + side;
      const long long lead = T.piece[q];
      if (lead < 2 * tb || lead >= 2 * (tb + nt)) {
        bad = true;
        break;
      }
      if (lead == q) {
        if (npieces >= ns + 1) {
          bad = true;
          break;
        }
        node_rec[npieces] = (int)q;
        nodeof[q - 2 * tb] = npieces++;
      }
    }
  }
  if (bad || npieces != ns + 1) {
    set_error(C, POLYLLA_ERR_LIMIT, 67);
    P.pcnt[i] = 0;
    P.flen[i] = 0;
    return;
  }
  // 2. chords in increasing tip vertex (heapsort), merged from the largest down
  for (int r = ns / 2 - 1; r >= 0; --r) heap_sift(chord_b, chord_k, r, ns);
  for (int e = ns - 1; e > 0; --e) {
    int t = chord_b[0]; chord_b[0] = chord_b[e]; chord_b[e] = t;
    t = chord_k[0]; chord_k[0] = chord_k[e]; chord_k[e] = t;
    heap_sift(chord_b, chord_k, 0, e);
  }
  for (int v = 0; v < npieces; ++v) {
    uf[v] = v;
    pos[v] = v;
  }
  int nodes = npieces;
  for (int c = ns - 1; c >= 0 && !bad; --c) {
    const long long k = chord_k[c];
    const int na = nodeof[T.piece[2 * k] - 2 * tb];
    const int nb = nodeof[T.piece[2 * k + 1] - 2 * tb];
    int ra = na, rb = nb;
    while (uf[ra] != ra) ra = uf[ra] = uf[uf[ra]];
    while (uf[rb] != rb) rb = uf[rb] = uf[uf[rb]];
    if (ra == rb || nodes >= W) {
      bad = true;
      break;
    }
    const int u = nodes++;
    left[u] = pos[ra];
    right[u] = pos[rb];
    uf[rb] = ra;
    pos[ra] = u;
  }
  if (bad) {
    set_error(C, POLYLLA_ERR_LIMIT, 68);
    P.pcnt[i] = 0;
    P.flen[i] = 0;
    return;
  }
  // 3. leaf counts bottom-up, in-order starts top-down (the root is the last node)
  for (int v = 0; v < npieces; ++v) cnt[v] = 1;
  for (int u = npieces; u < nodes; ++u) cnt[u] = cnt[left[u]] + cnt[right[u]];
  pos[nodes - 1] = 0;
  for (int u = nodes - 1; u >= npieces; --u) {
    pos[left[u]] = pos[u];
    pos[right[u]] = pos[u] + cnt[left[u]];
  }
  // 4. final piece slots
  const long long base = (long long)atomicAdd(
      reinterpret_cast<unsigned long long*>(&C->piece_alloc), (unsigned long long)npieces);
  if (base + npieces > F.cap) {
    set_error(C, POLYLLA_ERR_LIMIT, 69);
    P.pcnt[i] = 0;
    P.flen[i] = 0;
    return;
  }
  long long total = 0;
  for (int v = 0; v < npieces; ++v) {
    const int rec = node_rec[v];
    F.start[base + pos[v]] = T.rec_start[rec];
    F.len[base + pos[v]] = T.rec_len[rec];
    F.src[base + pos[v]] = src;
    T.rec_slot[rec] = (int)(base + pos[v]);
    total += T.rec_len[rec];
  }
  P.pbase[i] = (int)base;
  P.pcnt[i] = npieces;
  P.flen[i] = (int)total;
}

}  // namespace polylla
