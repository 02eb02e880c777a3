// Host planner of the tiled FP32 sweep: the characteristic grid of Sec. 3 cut into per-tile pieces.
//
// Every characteristic of an azimuth pair is walked by two senses; each sense's direction points into one
// quadrant.  Cutting the characteristic at tile boundaries gives pieces (a straight line meets a square tile at
// most once).  For a quadrant q and a tile, the geometry (tile, q) holds the pieces of every sense pointing into
// q that cross the tile, sorted longest first, so that the pieces still walking at step t are ranks 0 .. n_t - 1
// and the geometry's state and records are packed step by step (slot = P[t] + rank).  A piece hands its outgoing
// intensity to the next piece of its characteristic, in the next tile along its direction: the tile before a
// tile in x or in y (or, through a vertex, both), which therefore runs earlier in the quadrant's wavefront.
#include "molc_tiles.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace molc {

namespace {

inline int quadrant_of(double dx, double dy) { return (dx < 0 ? 1 : 0) | (dy < 0 ? 2 : 0); }

struct HostPiece {
  int track, sense, first, len, tile;
  int geom = -1, rank = -1;
};

}  // namespace

TileShape tile_shape(const TileTables &t, int n_pairs, int np) {
  TileShape sh;
  sh.max_item_floats = t.max_item_floats;
  sh.cd_entries = t.TS2p * t.GT;
  sh.max_len = t.max_len;
  sh.n_pairs = n_pairs;
  sh.split_units = t.max_split_units * t.GT;
  sh.np_exact = np;
  return sh;
}

size_t tile_smem_bytes(const TileTables &t, int n_pairs, int np) {
  return tile_sweep_smem(tile_shape(t, n_pairs, np), np);
}

namespace {

// Slots (piece segments) of the largest geometry for tile side TS, in one pass over the segments.
int64_t max_geometry_slots(const TilePlanInput &in, int TS, std::vector<int> &qp) {
  const int ntx = (in.nx + TS - 1) / TS, nty = (in.ny + TS - 1) / TS;
  std::vector<int64_t> cnt((size_t)4 * ntx * nty, 0);
  for (const TileTrack &tr : *in.tracks) {
    const int q0 = qp[2 * tr.pair], q1 = qp[2 * tr.pair + 1];
    for (int j = 0; j < tr.nseg; ++j) {
      const int c = in.seg_cell[tr.seg_off + j];
      const int tile = (c / in.nx) / TS * ntx + (c % in.nx) / TS;
      cnt[(size_t)q0 * ntx * nty + tile]++;
      cnt[(size_t)q1 * ntx * nty + tile]++;
    }
  }
  return *std::max_element(cnt.begin(), cnt.end());
}

bool build(const TilePlanInput &in, int TS, int GT, const std::vector<int> &qp, TileTables &t, std::string &why) {
  const int nx = in.nx, ny = in.ny, G = in.G, np = in.n_polar;
  t = TileTables();
  t.TS = TS;
  t.TS2p = (TS * TS + 3) / 4 * 4;
  t.ntx = (nx + TS - 1) / TS;
  t.nty = (ny + TS - 1) / TS;
  t.n_tiles = t.ntx * t.nty;
  t.n_geoms = 4 * t.n_tiles;
  t.GT = std::min(GT, G);
  t.n_gt = (G + t.GT - 1) / t.GT;
  t.n_items = t.n_gt * t.n_geoms;
  const std::vector<TileTrack> &tracks = *in.tracks;
  const int64_t T = (int64_t)tracks.size();
  auto tile_of = [&](int c) { return (c / nx) / TS * t.ntx + (c % nx) / TS; };
  auto local_of = [&](int c) { return ((c / nx) % TS) * TS + (c % nx) % TS; };

  // pieces of every (track, sense), in traversal order
  std::vector<HostPiece> pcs;
  std::vector<int64_t> ts_off((size_t)2 * T + 1, 0);
  std::vector<int64_t> ts_list;
  {
    std::vector<std::pair<int, int>> runs;   // (first, len) in + order
    for (int64_t k = 0; k < T; ++k) {
      const TileTrack &tr = tracks[k];
      runs.clear();
      int first = 0;
      for (int j = 1; j <= tr.nseg; ++j)
        if (j == tr.nseg || tile_of(in.seg_cell[tr.seg_off + j]) != tile_of(in.seg_cell[tr.seg_off + first])) {
          runs.emplace_back(first, j - first);
          first = j;
        }
      for (int sense = 0; sense < 2; ++sense) {
        ts_off[2 * k + sense] = (int64_t)ts_list.size();
        for (size_t r = 0; r < runs.size(); ++r) {
          const auto &run = sense ? runs[runs.size() - 1 - r] : runs[r];
          HostPiece hp;
          hp.track = (int)k;
          hp.sense = sense;
          hp.first = run.first;
          hp.len = run.second;
          hp.tile = tile_of(in.seg_cell[tr.seg_off + run.first]);
          ts_list.push_back((int64_t)pcs.size());
          pcs.push_back(hp);
        }
      }
    }
    ts_off[2 * T] = (int64_t)ts_list.size();
  }
  t.n_pieces = (int64_t)pcs.size();
  if (t.n_pieces >= ((int64_t)1 << 31) - 1) {
    why = "too many characteristic pieces";
    return false;
  }
  // geometries: bucket the pieces, longest first (ties in creation order: pair, track, sense)
  std::vector<std::vector<int64_t>> bucket(t.n_geoms);
  for (int64_t i = 0; i < (int64_t)pcs.size(); ++i) {
    const HostPiece &hp = pcs[i];
    const int q = qp[2 * tracks[hp.track].pair + hp.sense];
    bucket[(size_t)q * t.n_tiles + hp.tile].push_back(i);
  }
  t.geoms.resize(t.n_geoms);
  int64_t piece_off = 0, slot_base = 0, ent_off = 0;
  std::vector<std::vector<std::pair<int, std::pair<int, int>>>> cell_ents((size_t)TS * TS);  // (pair, (slot, af))
  for (int gidx = 0; gidx < t.n_geoms; ++gidx) {
    auto &b = bucket[gidx];
    std::stable_sort(b.begin(), b.end(), [&](int64_t x, int64_t y) { return pcs[x].len > pcs[y].len; });
    TileGeom &gm = t.geoms[gidx];
    gm.q = gidx / t.n_tiles;
    gm.tile = gidx % t.n_tiles;
    gm.n_pieces = (int)b.size();
    gm.max_len = b.empty() ? 0 : pcs[b[0]].len;
    gm.piece_off = piece_off;
    gm.slot_base = slot_base;
    gm.P_off = (int)t.Ptab.size();
    for (size_t r = 0; r < b.size(); ++r) {
      pcs[b[r]].geom = gidx;
      pcs[b[r]].rank = (int)r;
    }
    // P[t]: slots before step t
    std::vector<int> P(gm.max_len + 1, 0);
    {
      size_t alive = b.size();
      for (int s = 0; s < gm.max_len; ++s) {
        while (alive > 0 && pcs[b[alive - 1]].len <= s) --alive;
        P[s + 1] = P[s] + (int)alive;
      }
    }
    gm.n_slots = P[gm.max_len];
    if (gm.n_slots >= (1 << 24)) {
      why = "a tile holds too many piece segments";
      return false;
    }
    t.Ptab.insert(t.Ptab.end(), P.begin(), P.end());
    t.max_len = std::max(t.max_len, gm.max_len);
    // records and moment entries
    t.recs.resize((size_t)(slot_base + gm.n_slots));
    for (auto &ce : cell_ents) ce.clear();
    for (size_t r = 0; r < b.size(); ++r) {
      const HostPiece &hp = pcs[b[r]];
      const TileTrack &tr = tracks[hp.track];
      for (int s = 0; s < hp.len; ++s) {
        const int64_t seg = tr.seg_off + (hp.sense ? hp.first + hp.len - 1 - s : hp.first + s);
        const int c = in.seg_cell[seg];
        const int slot = P[s] + (int)r;
        const float lf = (float)in.seg_len[seg];
        const float af = (float)in.seg_afrac[seg];
        int lb, ab;
        std::memcpy(&lb, &lf, 4);
        std::memcpy(&ab, &af, 4);
        t.recs[(size_t)(slot_base + slot)] = make_int2(local_of(c), lb);
        cell_ents[local_of(c)].push_back({tr.pair, {slot, ab}});
      }
    }
    gm.ent_off = ent_off;
    gm.unit_off = (int)t.units.size();
    gm.cu_off = (int)t.cell_units.size();
    int split_units = 0;
    for (int cl = 0; cl < TS * TS; ++cl) {
      auto &ce = cell_ents[cl];
      std::stable_sort(ce.begin(), ce.end(), [](const std::pair<int, std::pair<int, int>> &x,
                                                const std::pair<int, std::pair<int, int>> &y) {
        return x.first < y.first || (x.first == y.first && x.second.first < y.second.first);
      });
      const int e0 = (int)(ent_off - gm.ent_off);
      for (auto &e : ce) t.ents.push_back(make_int2(e.second.first | (e.first << 24), e.second.second));
      ent_off += (int64_t)ce.size();
      const int n = (int)ce.size();
      const int parts = (n + kTileUnitEntries - 1) / kTileUnitEntries;
      t.cell_units.push_back(make_int2((int)t.units.size() - gm.unit_off, parts));
      for (int k = 0; k < parts; ++k)
        t.units.push_back(make_int4(cl, e0 + k * kTileUnitEntries, e0 + std::min(n, (k + 1) * kTileUnitEntries),
                                    0));
      if (parts > 1) split_units += parts;
    }
    gm.n_units = (int)t.units.size() - gm.unit_off;
    // the kernel keeps the partial sums of every unit of a geometry that has split cells
    if (split_units > 0) t.max_split_units = std::max(t.max_split_units, gm.n_units);
    // upstream geometries and wavefront step
    const int tx = gm.tile % t.ntx, ty = gm.tile / t.ntx;
    const int sx = (gm.q & 1) ? -1 : 1, sy = (gm.q & 2) ? -1 : 1;
    const int ux = tx - sx, uy = ty - sy;
    gm.up_x = (ux >= 0 && ux < t.ntx) ? gm.q * t.n_tiles + ty * t.ntx + ux : -1;
    gm.up_y = (uy >= 0 && uy < t.nty) ? gm.q * t.n_tiles + uy * t.ntx + tx : -1;
    gm.delta = (sx > 0 ? tx : t.ntx - 1 - tx) + (sy > 0 ? ty : t.nty - 1 - ty);
    piece_off += (int64_t)b.size();
    slot_base += gm.n_slots;
  }
  // pieces with their links: a piece receives through its own index, sends to the next piece's index
  t.pieces.assign((size_t)t.n_pieces, make_int4(0, 0, 0, 0));
  t.tpiece.resize((size_t)t.n_pieces);
  t.tpiece_off.assign(ts_off.begin(), ts_off.end());
  for (int64_t k = 0; k < T; ++k)
    for (int sense = 0; sense < 2; ++sense) {
      const int64_t a = ts_off[2 * k + sense], z = ts_off[2 * k + sense + 1];
      int step = 0;
      for (int64_t i = a; i < z; ++i) {
        const HostPiece &hp = pcs[ts_list[i]];
        const TileGeom &gm = t.geoms[hp.geom];
        const int64_t gi = gm.piece_off + hp.rank;
        int in_link = (int)gi;
        if (i == a) in_link = -1 - (sense ? tracks[k].entry_minus : tracks[k].entry_plus);
        int out_link = -1;
        if (i + 1 < z) {
          const HostPiece &nx_ = pcs[ts_list[i + 1]];
          out_link = (int)(t.geoms[nx_.geom].piece_off + nx_.rank);
        }
        t.pieces[(size_t)gi] = make_int4((int)k, 2 * hp.len + sense, in_link, out_link);
        t.tpiece[(size_t)i] = make_int4(hp.geom, hp.rank, step, 0);
        step += hp.len;
      }
    }
  // items in wavefront order (the groups of one geometry together), state offsets in that order
  std::vector<int> order((size_t)t.n_items);
  for (int i = 0; i < t.n_items; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const TileGeom &gx = t.geoms[x % t.n_geoms], &gy = t.geoms[y % t.n_geoms];
    if (gx.delta != gy.delta) return gx.delta < gy.delta;
    if (x % t.n_geoms != y % t.n_geoms) return x % t.n_geoms < y % t.n_geoms;
    return x / t.n_geoms < y / t.n_geoms;
  });
  t.queue = order;
  t.item_off.assign((size_t)t.n_items, 0);
  int64_t off = 0;
  for (int item : order) {
    const int gt = item / t.n_geoms, geom = item % t.n_geoms;
    const int gcount = std::min(t.GT, G - gt * t.GT);
    const int64_t floats = ((int64_t)t.geoms[geom].n_slots * gcount * np + 3) / 4 * 4;
    t.item_off[(size_t)item] = off;
    off += floats;
    t.max_item_floats = std::max<int64_t>(t.max_item_floats, floats);
  }
  t.state_floats = off;
  return true;
}

}  // namespace

bool check_tiles(const TilePlanInput &in, const TileTables &t, std::string &why) {
  auto bad = [&](const char *what) {
    why = std::string("tiled layout check failed: ") + what;
    return false;
  };
  const std::vector<TileTrack> &tracks = *in.tracks;
  const int64_t T = (int64_t)tracks.size();
  const int TS = t.TS, nx = in.nx;
  auto tile_of = [&](int c) { return (c / nx) / TS * t.ntx + (c % nx) / TS; };
  auto local_of = [&](int c) { return ((c / nx) % TS) * TS + (c % nx) % TS; };
  std::vector<int> qp((size_t)2 * in.n_pairs);
  for (int j = 0; j < in.n_pairs; ++j) {
    qp[2 * j] = quadrant_of(in.pair_c[j], in.pair_s[j]);
    qp[2 * j + 1] = quadrant_of(-in.pair_c[j], -in.pair_s[j]);
  }
  // every slot of every geometry is written by exactly one (piece, step), with that segment's record
  std::vector<uint8_t> seen(t.recs.size(), 0);
  for (int64_t k = 0; k < T; ++k)
    for (int sense = 0; sense < 2; ++sense) {
      const TileTrack &tr = tracks[k];
      const int64_t a = t.tpiece_off[2 * k + sense], z = t.tpiece_off[2 * k + sense + 1];
      int step = 0;
      for (int64_t i = a; i < z; ++i) {
        const int4 tp = t.tpiece[i];
        const TileGeom &gm = t.geoms[tp.x];
        const int64_t gi = gm.piece_off + tp.y;
        const int4 pc = t.pieces[gi];
        const int len = pc.y >> 1;
        if (pc.x != k || (pc.y & 1) != sense || tp.z != step) return bad("piece identity");
        if (gm.q != qp[2 * tr.pair + sense]) return bad("piece quadrant");
        for (int s = 0; s < len; ++s) {
          const int st = step + s;
          const int64_t seg = tr.seg_off + (sense ? tr.nseg - 1 - st : st);
          const int c = in.seg_cell[seg];
          if (tile_of(c) != gm.tile) return bad("segment outside its piece's tile");
          const int64_t slot = gm.slot_base + t.Ptab[gm.P_off + s] + tp.y;
          if (slot >= gm.slot_base + gm.n_slots || seen[slot]) return bad("record slot");
          seen[slot] = 1;
          const float lf = (float)in.seg_len[seg];
          int lb;
          std::memcpy(&lb, &lf, 4);
          if (t.recs[slot].x != local_of(c) || t.recs[slot].y != lb) return bad("record contents");
        }
        // links: entering from the boundary or from the previous piece; leaving to the next piece
        const int want_in = i == a ? -1 - (sense ? tr.entry_minus : tr.entry_plus) : (int)gi;
        if (pc.z != want_in) return bad("piece entry link");
        if (i + 1 < z) {
          const int4 tn = t.tpiece[i + 1];
          const TileGeom &gn = t.geoms[tn.x];
          if (pc.w != (int)(gn.piece_off + tn.y)) return bad("piece exit link");
          // the next tile lies one step along the direction: after this one in the quadrant's wavefront
          const int dx = gn.tile % t.ntx - gm.tile % t.ntx, dy = gn.tile / t.ntx - gm.tile / t.ntx;
          const int sx = (gm.q & 1) ? -1 : 1, sy = (gm.q & 2) ? -1 : 1;
          if (!((dx == 0 || dx == sx) && (dy == 0 || dy == sy) && (dx != 0 || dy != 0)) || gn.q != gm.q)
            return bad("consecutive pieces not in adjacent tiles along the direction");
          if (gn.delta <= gm.delta) return bad("wavefront order");
        } else if (pc.w != -1) {
          return bad("last piece has an exit link");
        }
        step += len;
      }
      if (step != tr.nseg) return bad("pieces do not cover the characteristic");
    }
  for (size_t i = 0; i < seen.size(); ++i)
    if (!seen[i]) return bad("unwritten record slot");
  // moment entries: every slot once, in the cell of its record; units cover each cell's entries
  std::fill(seen.begin(), seen.end(), 0);
  for (const TileGeom &gm : t.geoms) {
    const int TS2 = TS * TS;
    int64_t covered = 0;
    for (int cl = 0; cl < TS2; ++cl) {
      const int2 cu = t.cell_units[gm.cu_off + cl];
      int prev_end = -1;
      for (int u = 0; u < cu.y; ++u) {
        const int4 un = t.units[gm.unit_off + cu.x + u];
        if (un.x != cl || (prev_end >= 0 && un.y != prev_end) || un.z <= un.y) return bad("moment units");
        for (int e = un.y; e < un.z; ++e) {
          const int2 en = t.ents[gm.ent_off + e];
          const int slot = en.x & 0xFFFFFF;
          if (slot >= gm.n_slots || seen[gm.slot_base + slot]) return bad("moment entry slot");
          seen[gm.slot_base + slot] = 1;
          if (t.recs[gm.slot_base + slot].x != cl) return bad("moment entry cell");
          ++covered;
        }
        prev_end = un.z;
      }
    }
    if (covered != gm.n_slots) return bad("moment entries do not cover the geometry");
    // upstream geometries
    const int tx = gm.tile % t.ntx, ty = gm.tile / t.ntx;
    const int sx = (gm.q & 1) ? -1 : 1, sy = (gm.q & 2) ? -1 : 1;
    const int ux = tx - sx, uy = ty - sy;
    if (gm.up_x != (ux >= 0 && ux < t.ntx ? gm.q * t.n_tiles + ty * t.ntx + ux : -1)) return bad("upstream x");
    if (gm.up_y != (uy >= 0 && uy < t.nty ? gm.q * t.n_tiles + uy * t.ntx + tx : -1)) return bad("upstream y");
  }
  // queue: every item once, each after its upstream items; state ranges disjoint and 16-byte aligned
  std::vector<int> pos((size_t)t.n_items, -1);
  for (size_t i = 0; i < t.queue.size(); ++i) {
    if (t.queue[i] < 0 || t.queue[i] >= t.n_items || pos[t.queue[i]] >= 0) return bad("queue");
    pos[t.queue[i]] = (int)i;
  }
  int64_t end = 0;
  for (size_t i = 0; i < t.queue.size(); ++i) {
    const int item = t.queue[i], gt = item / t.n_geoms, g = item % t.n_geoms;
    const TileGeom &gm = t.geoms[g];
    for (int up : {gm.up_x, gm.up_y})
      if (up >= 0 && pos[gt * t.n_geoms + up] >= (int)i) return bad("queue order");
    if (t.item_off[item] != end || t.item_off[item] % 4) return bad("state offsets");
    const int gcount = std::min(t.GT, in.G - gt * t.GT);
    end += ((int64_t)gm.n_slots * gcount * in.n_polar + 3) / 4 * 4;
  }
  if (end != t.state_floats) return bad("state size");
  return true;
}

bool plan_tiles(const TilePlanInput &in, TileTables &t, std::string &why, int force_ts, int force_gt) {
  if (in.n_pairs > 256) {
    why = "more than 256 azimuth pairs";
    return false;
  }
  std::vector<int> qp((size_t)2 * in.n_pairs);
  for (int j = 0; j < in.n_pairs; ++j) {
    qp[2 * j] = quadrant_of(in.pair_c[j], in.pair_s[j]);
    qp[2 * j + 1] = quadrant_of(-in.pair_c[j], -in.pair_s[j]);
  }
  const int np = in.n_polar;
  const size_t budget = kTileStateBytes;
  for (int TS : kTileCandidates) {
    if (force_ts > 0 && TS != force_ts) continue;
    if (TS > 1 && TS > std::max(in.nx, in.ny) && force_ts <= 0) continue;   // one tile already holds the grid
    const int64_t slots = max_geometry_slots(in, TS, qp);
    if ((size_t)slots * np * sizeof(float) > budget && force_ts <= 0) continue;
    for (int GT : kTileGroupCandidates) {
      if (force_gt > 0 && GT != force_gt) continue;
      if (GT > in.G && GT > 1) continue;
      if ((size_t)slots * std::min(GT, in.G) * np * sizeof(float) > budget) continue;
      if (!build(in, TS, GT, qp, t, why)) return false;
      if ((int64_t)t.max_split_units * t.GT > kTileMaxUnits) continue;
      if (tile_smem_bytes(t, in.n_pairs, np) > 224 * 1024) continue;   // below the opt-in limit of a block
      return check_tiles(in, t, why);
    }
  }
  why = "no tile size keeps a work item's state within the shared-memory budget";
  return false;
}

}  // namespace molc
