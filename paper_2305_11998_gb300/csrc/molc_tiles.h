// Host planner of the tiled FP32 sweep (molc_tiles.cpp): cuts the characteristic grid of a plan into per-tile
// pieces and builds the tables the tiled kernels read (see TileGeom / TileView in molc_internal.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "molc_internal.h"

namespace molc {

struct TileTrack {      // one characteristic of an azimuth pair, segments [seg_off, seg_off + nseg) in + order
  int64_t seg_off;
  int nseg, pair, entry_plus, entry_minus;
};

struct TilePlanInput {
  int nx, ny, G, n_pairs, n_polar;
  const double *pair_c, *pair_s;   // unit in-plane direction of each pair's + sense
  const std::vector<TileTrack> *tracks;
  const int *seg_cell;
  const double *seg_len, *seg_afrac;
};

struct TileTables {     // host copies of a tiled layout
  int TS = 0, TS2p = 0, ntx = 0, nty = 0, n_tiles = 0, n_geoms = 0, GT = 0, n_gt = 0, n_items = 0;
  int max_item_floats = 0, max_len = 0, max_split_units = 0;
  int64_t state_floats = 0, n_pieces = 0;
  std::vector<TileGeom> geoms;
  std::vector<int> Ptab;
  std::vector<int4> pieces;
  std::vector<int2> recs, ents, cell_units;
  std::vector<int4> units;
  std::vector<int64_t> item_off;
  std::vector<int> queue;          // item ids in wavefront order
  std::vector<int4> tpiece;        // per (track, sense), pieces in traversal order: {geom, rank, first step, 0}
  std::vector<int64_t> tpiece_off; // [2 T + 1]: range of (track k, sense s) = [off[2k+s], off[2k+s+1])
};

// Shared-memory shape and bytes of one tiled-sweep block for a layout.
TileShape tile_shape(const TileTables &t, int n_pairs, int np);
size_t tile_smem_bytes(const TileTables &t, int n_pairs, int np);

// Choose the tile size and groups per item (the largest tile whose items fit the shared-memory budget, then the
// most groups per item that still fit) and build the tables.  force_ts / force_gt > 0 pin a choice (autotuner).
// Returns false with a message when no candidate fits.
bool plan_tiles(const TilePlanInput &in, TileTables &t, std::string &why, int force_ts = 0, int force_gt = 0);

// Checks every invariant the tiled kernels rely on (run by plan_tiles on each layout it returns): each segment of
// each sense is one record slot with its cell and length, pieces cover their characteristic in traversal order,
// consecutive pieces lie in adjacent tiles along the direction and later in the quadrant's wavefront, links chain
// them, moment entries and units cover every slot once in its record's cell, the queue lists every item after
// its upstream items, and item states are disjoint 16-byte aligned ranges.  False with a message otherwise.
bool check_tiles(const TilePlanInput &in, const TileTables &t, std::string &why);

}  // namespace molc
