"""Seeded synthetic inputs shared by the CUDA path tests, the oracle tests and bench.py.

This module holds no arithmetic of the Coulomb method itself: no quadrature, no tables,
no integral values.  It only draws random numbers and turns them into the inputs the
engine consumes:

* the planewave index set of a cutoff sphere |n|^2 <= R^2 (the input basis; Sec. III of
  the paper enumerates it only by its shell-closing counts) and a dense cube -> id map
  that lets the generator name the fourth function of a drawn quadruple;
* quadruples (I, J, K, L) of basis ids, drawn uniformly over the basis and completed so
  that n_L = n_I + n_K - n_J lies in the sphere (rejection, bounded attempts);
* the per-box parameters of the batched workload.

All randomness is counter-based SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): output number c of a generator started at
state k is mix64(k + (c + 1) * GAMMA).  Every draw is a pure function of
(seed, stream, counter), so any quadruple can be regenerated on its own, on the host or
on the device (the CUDA twin lives in coulomb_inputs/gen.cu and is tested for bit
equality against this file).
"""
from __future__ import annotations

import numpy as np

SEED = 150208043
GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

# attempts per quadruple before the deterministic fallback (I, I, K, K); with an
# acceptance of about 0.32 the fallback has probability 0.68**64 ~ 2e-11 per quadruple
ATTEMPTS = 64

# quadruple streams
STREAM_CLEAN = 1        # only momentum-conserving quadruples
STREAM_PLANTED = 2      # 5 % random L (non-conserving), 1 % I = J, L = K
STREAM_UNIFORM = 3      # four independent uniform ids (almost all non-conserving)


def _u64(x):
    return np.asarray(x, dtype=np.uint64)


def mix64(z):
    """SplitMix64 finaliser on uint64 arrays (wrap-around arithmetic)."""
    z = _u64(z)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
        z = z ^ (z >> np.uint64(31))
    return z


def stream_key(seed: int, stream: int) -> int:
    """Starting state of stream `stream` under `seed` (a python int < 2**64)."""
    return int(mix64(np.uint64((seed + (stream + 1) * GAMMA) & MASK64)))


def draw(key: int, ctr):
    """Counter-th SplitMix64 output of the generator whose state starts at `key`."""
    ctr = _u64(ctr)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(key) + (ctr + np.uint64(1)) * np.uint64(GAMMA))


def lemire(u64, n: int):
    """Map the top 32 bits of a 64-bit draw onto [0, n) by multiply-high (Lemire 2019)."""
    hi = _u64(u64) >> np.uint64(32)
    return ((hi * np.uint64(n)) >> np.uint64(32)).astype(np.int64)


def uniform01(u64):
    """Top 53 bits of a draw as a double in [0, 1)."""
    return (_u64(u64) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# --------------------------------------------------------------------------------------
# input basis: integer vectors of a cutoff sphere, lexicographic (n_x, n_y, n_z) order
# --------------------------------------------------------------------------------------
def sphere_vectors(R: int) -> np.ndarray:
    r = np.arange(-R, R + 1)
    X, Y, Z = np.meshgrid(r, r, r, indexing="ij")
    keep = (X * X + Y * Y + Z * Z) <= R * R
    return np.stack([X[keep], Y[keep], Z[keep]], axis=1).astype(np.int64)


def cube_id_map(R: int, vec: np.ndarray) -> np.ndarray:
    """Dense (2R+1)^3 map from an integer vector to its id in `vec`, -1 outside."""
    G = 2 * R + 1
    m = np.full(G * G * G, -1, dtype=np.int32)
    idx = ((vec[:, 0] + R) * G + (vec[:, 1] + R)) * G + (vec[:, 2] + R)
    m[idx] = np.arange(len(vec), dtype=np.int32)
    return m


def quads(R: int, start: int, count: int, seed: int = SEED, stream: int = STREAM_CLEAN,
          vec: np.ndarray | None = None, idmap: np.ndarray | None = None,
          indices=None) -> np.ndarray:
    """Quadruples number start .. start+count-1 of `stream` (or the quadruple numbers in
    `indices`, when given), as int32[count, 4] ids.

    Quadruple i, attempt a, component c (0: I, 1: J, 2: K, 3: planting) uses counter
    (i * ATTEMPTS + a) * 4 + c.  I, J, K are uniform ids; L is the id of
    n_I + n_K - n_J when that vector lies in the sphere, else the next attempt is taken.
    """
    if vec is None:
        vec = sphere_vectors(R)
    if idmap is None:
        idmap = cube_id_map(R, vec)
    Nb = len(vec)
    G = 2 * R + 1
    key = stream_key(seed, stream)
    if indices is not None:
        i = np.asarray(indices, dtype=np.uint64)
        count = len(i)
    else:
        i = np.arange(start, start + count, dtype=np.uint64)
    out = np.empty((count, 4), dtype=np.int32)
    done = np.zeros(count, dtype=bool)
    first = None
    for a in range(ATTEMPTS):
        todo = np.nonzero(~done)[0]
        if todo.size == 0:
            break
        base = (i[todo] * np.uint64(ATTEMPTS) + np.uint64(a)) * np.uint64(4)
        I = lemire(draw(key, base), Nb)
        J = lemire(draw(key, base + np.uint64(1)), Nb)
        K = lemire(draw(key, base + np.uint64(2)), Nb)
        if a == 0:
            first = (I.copy(), K.copy())
        nL = vec[I] + vec[K] - vec[J]
        ok = (nL * nL).sum(axis=1) <= R * R
        nLc = np.clip(nL + R, 0, G - 1)
        Lid = idmap[(nLc[:, 0] * G + nLc[:, 1]) * G + nLc[:, 2]]
        sel = todo[ok]
        out[sel, 0] = I[ok]
        out[sel, 1] = J[ok]
        out[sel, 2] = K[ok]
        out[sel, 3] = Lid[ok]
        done[sel] = True
    if not done.all():  # deterministic fallback (I, I, K, K) from attempt 0
        rest = np.nonzero(~done)[0]
        I0, K0 = first  # attempt 0 drew every quadruple, so index directly
        out[rest, 0] = I0[rest]
        out[rest, 1] = I0[rest]
        out[rest, 2] = K0[rest]
        out[rest, 3] = K0[rest]
    if stream == STREAM_PLANTED:
        b0 = i * np.uint64(ATTEMPTS) * np.uint64(4) + np.uint64(3)
        u = (draw(key, b0) >> np.uint64(32)).astype(np.int64)
        rnd = lemire(draw(key, b0 + np.uint64(4)), Nb)
        nonc = u < int(0.05 * 2 ** 32)
        same = (~nonc) & (u < int(0.06 * 2 ** 32))
        out[nonc, 3] = rnd[nonc]
        out[same, 1] = out[same, 0]
        out[same, 3] = out[same, 2]
    return out


def quads_uniform(R: int, start: int, count: int, seed: int = SEED,
                  stream: int = STREAM_UNIFORM) -> np.ndarray:
    """Quadruples number start .. start+count-1 with four independent uniform ids, as
    int32[count, 4]: component c of quadruple i uses counter 4 i + c.  The inputs of
    general (not necessarily momentum-conserving) integrals."""
    Nb = len(sphere_vectors(R))
    key = stream_key(seed, stream)
    i = np.arange(start, start + count, dtype=np.uint64)
    out = np.empty((count, 4), dtype=np.int32)
    for c in range(4):
        out[:, c] = lemire(draw(key, i * np.uint64(4) + np.uint64(c)), Nb)
    return out


def quads_as_vectors(q: np.ndarray, vec: np.ndarray) -> np.ndarray:
    """The int8x4 form of id quadruples: int8[count, 4 functions, 4] = (n_x, n_y, n_z, 0)."""
    out = np.zeros((q.shape[0], 4, 4), dtype=np.int8)
    out[:, :, :3] = vec[q].astype(np.int8)
    return out


# --------------------------------------------------------------------------------------
# batched workload: 256 independent boxes with uneven cutoffs, sides, radii, node counts
# --------------------------------------------------------------------------------------
STREAM_BOXES = 1000


def box_params(nbox: int = 256, seed: int = SEED):
    """Per box b: R in 4..24, L in [8, 30) bohr, R_F = max(1, round((0.4 + 0.4u) R)),
    S in 16..96, each from its own uniform draw u of stream STREAM_BOXES + b."""
    boxes = []
    for b in range(nbox):
        key = stream_key(seed, STREAM_BOXES + b)
        u = uniform01(draw(key, np.arange(4, dtype=np.uint64)))
        R = 4 + int(np.floor(21 * u[0]))
        L = 8.0 + 22.0 * float(u[1])
        RF = max(1, int(np.rint((0.4 + 0.4 * u[2]) * R)))
        S = 16 + int(np.floor(81 * u[3]))
        boxes.append({"R": R, "L": L, "R_F": RF, "S": S})
    return boxes


# --------------------------------------------------------------------------------------
# device twin (coulomb_inputs/gen.cu -> libccgen.so): same quadruples, generated on the GPU
# --------------------------------------------------------------------------------------
_GEN_LIB = None
_GEN_TABLES = {}


def _gen_lib():
    global _GEN_LIB
    if _GEN_LIB is None:
        import ctypes
        import os
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libccgen.so")
        if not os.path.exists(path):
            raise ImportError("coulomb_inputs/libccgen.so is not built (run the package build)")
        L = ctypes.CDLL(path)
        P, I, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
        L.ccgen_quads.restype = I
        L.ccgen_quads.argtypes = [I, I, P, P, ctypes.c_ulonglong, LL, LL, I, P, P]
        _GEN_LIB = L
    return _GEN_LIB


def quads_device(R: int, start: int, count: int, out, seed: int = SEED,
                 stream: int = STREAM_CLEAN, cuda_stream=None):
    """Fill the int32[count, 4] CUDA tensor `out` with quadruples start .. start+count-1,
    bit-identical to quads(R, start, count, seed, stream) (quads_uniform for
    STREAM_UNIFORM)."""
    import torch
    dev = out.device
    key_t = (R, dev.index)
    if key_t not in _GEN_TABLES:
        vec = sphere_vectors(R)
        v4 = np.zeros((len(vec), 4), dtype=np.int8)
        v4[:, :3] = vec
        _GEN_TABLES[key_t] = (torch.from_numpy(v4).to(dev), torch.from_numpy(cube_id_map(R, vec)).to(dev),
                              len(vec))
    v4, idm, Nb = _GEN_TABLES[key_t]
    assert out.dtype == torch.int32 and out.is_contiguous() and out.shape[0] >= count
    s = torch.cuda.current_stream(dev).cuda_stream if cuda_stream is None else cuda_stream
    rc = _gen_lib().ccgen_quads(R, Nb, v4.data_ptr(), idm.data_ptr(), stream_key(seed, stream),
                                start, count,
                                {STREAM_PLANTED: 1, STREAM_UNIFORM: 2}.get(stream, 0),
                                out.data_ptr(), s)
    if rc != 0:
        raise RuntimeError(f"ccgen_quads failed ({rc})")
    return out
