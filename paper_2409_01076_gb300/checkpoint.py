"""Checkpoint files of a single lattice: a fixed 96-byte header and the canonical f(t).

File layout (little-endian):

    offset  size  field
         0     8  magic b"SMRTCKP1"
         8     4  int32   nx
        12     4  int32   ny
        16     8  float64 tau
        24     8  float64 u_lid
        32     8  float64 tau_s
        40     4  uint32  bc_flags
        44     4  int32   precision   (SMRT_PREC_*)
        48     4  int32   layout      (SMRT_LAYOUT_*)
        52     4  int32   collision   (SMRT_COLLISION_*)
        56     8  int64   t           (updates applied so far)
        64     4  int32   rounding    (SMRT_ROUND_*; 0 in files written before the option existed)
        68    28  reserved, zero
        96     -  float64 f[9][ny][nx], the canonical f(t) of smrt_get_f

Resuming from a file is bit for bit the same as running straight through for 32- and 16-bit storage
(the export f = g + w rounds back to the stored offset g exactly) and within one double ulp of the
offset for FP64 storage.  The file holds no device pointer and no build information: any build of the
library reads it.
"""
from __future__ import annotations

import struct

import numpy as np

MAGIC = b"SMRTCKP1"
HEADER = struct.Struct("<8s2i3dI3iqi28x")
assert HEADER.size == 96

_FIELDS = ("nx", "ny", "tau", "u_lid", "tau_s", "bc", "precision", "layout", "collision", "t", "rounding")


def write_checkpoint(path: str, header: dict, f: np.ndarray) -> None:
    """Writes `header` (the keys of _FIELDS) and f (float64, shape (9, ny, nx)) to path."""
    f = np.ascontiguousarray(f, dtype="<f8")
    if f.shape != (9, header["ny"], header["nx"]):
        raise ValueError("f has shape %s, the header says (9, %d, %d)" % (f.shape, header["ny"], header["nx"]))
    with open(path, "wb") as fh:
        fh.write(HEADER.pack(MAGIC, *(header.get(k, 0) if k == "rounding" else header[k] for k in _FIELDS)))
        fh.write(f.tobytes())


def read_checkpoint(path: str):
    """(header dict, f) from a file written by write_checkpoint; ValueError if it is not one."""
    with open(path, "rb") as fh:
        raw = fh.read(HEADER.size)
        if len(raw) != HEADER.size:
            raise ValueError("%s: too short for a checkpoint header" % path)
        vals = HEADER.unpack(raw)
        if vals[0] != MAGIC:
            raise ValueError("%s: not an SmrtLBM checkpoint (magic %r)" % (path, vals[0]))
        header = dict(zip(_FIELDS, vals[1:]))
        nx, ny = header["nx"], header["ny"]
        if nx < 2 or ny < 2:
            raise ValueError("%s: bad lattice size %d x %d" % (path, nx, ny))
        f = np.fromfile(fh, dtype="<f8", count=9 * ny * nx)
        if f.size != 9 * ny * nx:
            raise ValueError("%s: %d of %d population values present" % (path, f.size, 9 * ny * nx))
    return header, f.reshape(9, ny, nx).astype(np.float64)


def save_checkpoint(h, path: str) -> None:
    """Writes the state of handle h (made by smrt_create) to path."""
    from . import (SMRT_OPT_COLLISION, SMRT_OPT_LAYOUT, SMRT_OPT_PRECISION, SMRT_OPT_ROUNDING, SMRT_OPT_TAU,
                   SMRT_OPT_TAU_S, smrt_get_f, smrt_get_option, smrt_time)
    f = np.empty((9, h.ny, h.nx), dtype=np.float64)
    smrt_get_f(h, f)
    header = {"nx": h.nx, "ny": h.ny, "tau": smrt_get_option(h, SMRT_OPT_TAU), "u_lid": h.u_lid,
              "tau_s": smrt_get_option(h, SMRT_OPT_TAU_S), "bc": h.bc,
              "precision": int(smrt_get_option(h, SMRT_OPT_PRECISION)),
              "layout": int(smrt_get_option(h, SMRT_OPT_LAYOUT)),
              "collision": int(smrt_get_option(h, SMRT_OPT_COLLISION)), "t": smrt_time(h),
              "rounding": int(smrt_get_option(h, SMRT_OPT_ROUNDING))}
    write_checkpoint(path, header, f)


def load_checkpoint(path: str):
    """A new handle in the state saved at path (same lattice, options, t and populations)."""
    from . import (SMRT_LAYOUT_AA, SMRT_OPT_COLLISION, SMRT_OPT_LAYOUT, SMRT_OPT_PRECISION, SMRT_OPT_ROUNDING,
                   SMRT_OPT_TAU_S, smrt_create, smrt_set_f, smrt_set_option, smrt_set_time, smrt_step)
    header, f = read_checkpoint(path)
    h = smrt_create(header["nx"], header["ny"], header["tau"], header["u_lid"], header["bc"])
    smrt_set_option(h, SMRT_OPT_PRECISION, header["precision"])
    smrt_set_option(h, SMRT_OPT_LAYOUT, header["layout"])
    smrt_set_option(h, SMRT_OPT_COLLISION, header["collision"])
    smrt_set_option(h, SMRT_OPT_TAU_S, header["tau_s"])
    smrt_set_option(h, SMRT_OPT_ROUNDING, header["rounding"])
    t = header["t"]
    if header["layout"] == SMRT_LAYOUT_AA and t % 2 == 1:
        smrt_step(h, 1)         # the in-place arrangement follows the parity of t: make it odd first
    smrt_set_f(h, f)
    smrt_set_time(h, t)
    return h
