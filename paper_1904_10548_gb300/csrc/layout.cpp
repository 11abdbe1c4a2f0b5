// Shared-memory layout of the persistent kernels on the host: team width
// and teams per block, the split of a block's shared memory into work
// buffers, and the layouts the library refuses before any launch.  Host
// code only (no CUDA calls), so that it can be checked on a machine
// without a GPU.
#include <algorithm>

#include "kernels.cuh"
#include "rn_internal.h"

namespace rn {

// Bytes of one team region: the block's shared memory (the opt-in limit, or
// the SM's share when several blocks must sit on one SM) less the
// reserved and static parts, the block header and the network copy, split
// among tpb teams (16-byte multiples).  Blocks per SM: enough for every
// item, at most what 128 registers a thread allow (the kernels' launch
// bound), at most 4.
int team_bytes_for(int sms, int optin, int per_sm, int reserved, int n_items, int tpb, int block,
                   int net_bytes, int static_smem, int *team_bytes, int *blocks_per_sm) {
  const int by_regs = std::max(1, 65536 / (block * 128));
  const int bpsm = std::max(1, std::min({4, by_regs, (n_items + sms - 1) / std::max(1, sms)}));
  const int budget = std::min(optin, per_sm / bpsm - reserved) - static_smem;
  const int tb = ((budget - kHdrBytes - net_bytes) / tpb) & ~15;
  if (blocks_per_sm) *blocks_per_sm = bpsm;
  if (tb <= 0) {
    set_error("shared memory: the network data leave no room for the work buffers");
    return RN_ERR_UNSUPPORTED;
  }
  *team_bytes = tb;
  return RN_OK;
}

// Work-buffer sizes of elements of eb bytes in team regions of team_bytes
// for teams of tw threads, tpb to a block: the team buffer holds the forward slots of
// `mode` (up to three per warp) and a backward segment (as
// many chain rows as fit, up to the longest chain); the group buffer (all
// regions) holds the group's descriptor, the rows of a whole group if
// they fit, and as many chain-head rows as the rest allows.
int layout_sizes(const Plan &p, const RowDims &f, int eb, int team_bytes, int net_bytes, int tw,
                 int tpb, int mode, Sizes *z) {
  const int misc = (int)round16((4 + 2 * kSeg) * sizeof(int));
  const int nw = tw / 32;
  z->tpb = tpb;
  z->team_bytes = team_bytes;
  z->net_bytes = net_bytes;
  z->buf = ((team_bytes - misc) & ~15) / eb - 72;
  z->gbuf = ((tpb * team_bytes - misc) & ~15) / eb - 72;
  z->fslots = 3;
  while (z->fslots > 1 && fwd_elems(nw, z->fslots, f.NXP, f.NUP, f.YP, f.SP, mode) > z->buf)
    --z->fslots;
  if (fwd_elems(nw, z->fslots, f.NXP, f.NUP, f.YP, f.SP, mode) > z->buf ||
      chain_back_elems(1, f.SP, f.NEP, f.NXP, f.NUP) > z->buf) {
    set_error("shared memory: the network is too large for the work buffers");
    return RN_ERR_UNSUPPORTED;
  }
  z->segb = 1;
  while (z->segb < p.max_chain_len &&
         chain_back_elems(z->segb + 1, f.SP, f.NEP, f.NXP, f.NUP) <= z->buf)
    ++z->segb;
  if (p.n_groups == 0) {
    z->gcap = 0;
    z->hchunk = 1;
    return RN_OK;
  }
  const int desc = round4((p.max_desc * 4 + eb - 1) / eb);
  z->fbrows = std::min(p.max_group, 64);
  const int rows = (z->gbuf - group_elems(0, 0, f.SP, f.NEP, z->fbrows, desc)) / f.SP;
  if (rows < 2) {
    set_error("shared memory: the network is too large for the group buffer");
    return RN_ERR_UNSUPPORTED;
  }
  // every group in shared memory if there is room beside one head row; a
  // larger group keeps all its rows in global memory
  const int wrows = p.n_roots > 0 ? p.max_root_children + 1 : 1;  // root_step work rows
  if (rows < 1 + wrows) {
    set_error("shared memory: the network is too large for the group buffer");
    return RN_ERR_UNSUPPORTED;
  }
  z->gcap = std::min(p.max_group, rows - wrows);
  z->hchunk = std::max(wrows, std::min(p.max_group_chains, rows - z->gcap));
  return RN_OK;
}

// Team width tw (one thread per input component, at least 64, a multiple
// of 32, at most 256), components per thread maxc (also ceil(nx / 32) for
// the per-node dual update: 1, 2, 4 or 8) and teams per block (four up to
// 512 threads: one block per SM, 16 warps for a group).
int team_layout(int block_threads, int nx, int nu, int *tw_out, int *tpb_out, int *maxc_out) {
  int tw = block_threads > 0 ? ((block_threads + 31) / 32) * 32
                             : std::max(64, ((std::max(nx, nu) + 31) / 32) * 32);
  tw = std::min(tw, 256);
  auto comps = [&](int b) {
    int c = std::max((std::max(nx, nu) + b - 1) / b, (nx + 31) / 32);
    return c <= 1 ? 1 : (c <= 2 ? 2 : (c <= 4 ? 4 : (c <= 8 ? 8 : 16)));
  };
  while (comps(tw) > 8 && tw < 256) tw += 32;
  if (comps(tw) > 8) {
    set_error("network: nx, nu too large for the team width");
    return RN_ERR_UNSUPPORTED;
  }
  *tw_out = tw;
  *tpb_out = tw <= 128 ? 4 : 2;
  if (maxc_out) *maxc_out = comps(tw);
  return RN_OK;
}

// Layout limits of the library: every work item has a resident block of
// its own, every group's rows fit in shared memory and all its chain heads
// are staged at once.  (The kernels carry code for blocks with several
// items, rows in global memory and chunked heads, but those paths are
// not validated on a GPU; such layouts are refused here, before launch.)
int check_layout(const Plan &p, const Sizes &z, int n_items, int grid, const char *what) {
  if (n_items > grid) {
    set_error("%s: %d work items exceed the %d resident blocks (fewer scenarios, or a "
              "smaller network, fit)", what, n_items, grid);
    return RN_ERR_UNSUPPORTED;
  }
  if (p.n_groups > 0 && (p.max_group > z.gcap || p.max_group_chains > z.hchunk)) {
    set_error("%s: a group of %d top nodes with %d chains exceeds the shared-memory "
              "capacity (%d rows, %d heads)", what, p.max_group, p.max_group_chains, z.gcap,
              z.hchunk);
    return RN_ERR_UNSUPPORTED;
  }
  return RN_OK;
}

}  // namespace rn
