"""Column-sharded back-transformation over several GPUs (one process per GPU).

Left multiplication by Q2 acts on every eigenvector column on its own, so
one problem's nev columns split over P ranks with no exchange during the
step (the paper distributes the same step over MPI ranks, Sec. 3 and 4; a
row distribution would need boundary rows passed between ranks every sweep,
a column distribution needs nothing):

* the reflectors are replicated: one broadcast from the rank that holds them
  (or every rank loads/produces them itself and skips the broadcast);
* rank r owns a contiguous block of columns, aligned to the tensor-core
  kernel's 128-column work items so that no item is split;
* every rank runs ``gb_trans_ev_tridi_to_band_d`` on its block;
* an optional all-gather assembles the whole Z on every rank afterwards.

This module only schedules and moves data; the arithmetic is the library's.
"""
import torch
import torch.distributed as dist

from . import _lib as gb

ITEM_COLUMNS = 128


def column_shard(nev, world, rank, align=ITEM_COLUMNS):
    """(first column, column count) of rank `rank` among `world` ranks:
    contiguous blocks of whole `align`-column units, as even as possible."""
    if world < 1 or not 0 <= rank < world or nev < 0:
        raise ValueError("bad shard arguments")
    units = (nev + align - 1) // align
    base, extra = divmod(units, world)
    u0 = rank * base + min(rank, extra)
    u1 = u0 + base + (1 if rank < extra else 0)
    c0, c1 = min(nev, u0 * align), min(nev, u1 * align)
    return c0, c1 - c0


def broadcast_reflectors(hh_v, hh_tau, src=0, group=None):
    """Replicate the reflector set from rank `src` (in place on the other
    ranks' tensors, which must have the same shapes)."""
    dist.broadcast(hh_v, src, group=group)
    dist.broadcast(hh_tau, src, group=group)


def _library_apply(n, nbw, hh_v, hh_tau, Zloc, opts=None, stream=None):
    """Z_loc <- Q2 Z_loc through the C ABI (device tensors, column-major)."""
    nloc = Zloc.shape[1]
    if nloc == 0:
        return gb.GB_OK
    ldz = Zloc.stride(1) if nloc > 1 else n
    ws_bytes = gb.gb_trans_ev_workspace_bytes(n, nbw, nloc, Zloc.is_complex(), opts)
    ws = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=Zloc.device)
    st = stream if stream is not None else torch.cuda.current_stream(Zloc.device)
    f = gb.gb_trans_ev_tridi_to_band_z if Zloc.is_complex() else gb.gb_trans_ev_tridi_to_band_d
    f(n, nbw, nloc, hh_v, hh_tau, Zloc, ldz, ws, ws_bytes, st, opts)
    return gb.gb_trans_ev_query(ws, ws_bytes, st)


def trans_ev_sharded(n, nbw, hh_v, hh_tau, Zloc, nev, group=None, src=None, gather=False, opts=None,
                     apply=None):
    """Back-transform this rank's column block of one problem.

    Zloc: this rank's columns (n x count, column-major: the transpose of a
    contiguous (count, n) tensor), count = column_shard(nev, P, rank)[1].
    src: if not None, the reflectors are broadcast from that rank first.
    gather: if True, returns the whole n x nev Z (every rank), else Zloc.
    apply: the per-rank compute, (n, nbw, hh_v, hh_tau, Zloc) -> status;
    the library call by default.
    Returns (Z, status)."""
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    c0, cnt = column_shard(nev, world, rank)
    if Zloc.shape[1] != cnt or Zloc.shape[0] < n:
        raise ValueError(f"rank {rank} holds {tuple(Zloc.shape)}, expected ({n}, {cnt}) columns {c0}..")
    if src is not None and world > 1:
        broadcast_reflectors(hh_v, hh_tau, src, group)
    if apply is None:
        status = _library_apply(n, nbw, hh_v, hh_tau, Zloc, opts)
    else:
        status = apply(n, nbw, hh_v, hh_tau, Zloc)
    if not gather or world == 1:
        return Zloc, status
    # all-gather of the column blocks (every block padded to the largest)
    counts = [column_shard(nev, world, r)[1] for r in range(world)]
    width = max(counts)
    pad = torch.zeros((width, n), dtype=Zloc.dtype, device=Zloc.device)
    pad[:cnt] = Zloc.T[:, :n]
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    Zt = torch.cat([p[:c] for p, c in zip(parts, counts)], dim=0)     # (nev, n): column-major n x nev
    return Zt.T, status
