"""Seeded synthetic serial chains and joint states.

The paper's experiments use randomly initialised robots (Section IV: the twists
and other configuration parameters are drawn at random) and randomised joint
inputs. This module draws such robots and states. It is input data only: it holds
none of the forward-dynamics arithmetic, and both the CPU oracle and the CUDA path
consume what it returns.

Conventions of the returned model (one chain = n links, joint i joins link i-1 to
link i, link 0 being the fixed base):

* ``axes[i]``      unit joint axis a_i of a revolute joint, in child frame i.
* ``frames[i]``    home transform parent -> child, 12 numbers: R (row-major 3x3)
                   then p (3); the joint transform is (R, p) * exp([a_i; 0] q_i).
* ``inertias[i]``  6x6 spatial inertia J_i at the origin of frame i, twist order
                   (omega; v):  [[I_c - m c^ c^, m c^], [-m c^, m 1]].
* ``offsets``      CSR offsets of the chains into the packed link arrays.

Distributions (one seed, drawn in this order for the whole batch of L links):
  1. axes      L x 3  standard normal, then normalised;
  2. lengths   L      U[0.1, 0.5] m  (home offset length, ``p = length * u``);
  3. dirs      L x 3  standard normal, normalised (direction u of the offset);
  4. masses    L      U[0.5, 5] kg;
  5. coms      L x 3  U[-0.05, 0.05] m (centre of mass in the link frame);
  6. moments   L x 3  U[0.01, 0.1] kg m^2, i.i.d. principal moments;
  7. quats     L x 4  standard normal, normalised: rotation of the principal axes;
  8. homerot   L x 4  standard normal, normalised (only drawn when
                       ``random_home_rotation``; else every home rotation is I).
States: q ~ U[-pi, pi], qdot ~ N(0, 1), tau ~ N(0, 10^2), drawn in that order.
Kinematic trees (``random_trees``): the same links, joined by a parent array
drawn from seed + 1 (``random_parents``: a link continues the previous link's
branch, or branches off a uniformly drawn earlier link with probability 0.3, or
starts on the base with probability 0.05).
Chain lengths for uneven batches: n = round(exp(U[ln lo, ln hi])) clamped to
[lo, hi].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

GRAVITY = np.array([0.0, 0.0, -9.81])


@dataclass
class ChainModel:
    axes: np.ndarray        # [L, 3]
    frames: np.ndarray      # [L, 12]
    inertias: np.ndarray    # [L, 36]
    offsets: np.ndarray     # [K + 1] int64
    gravity: np.ndarray     # [3]
    parents: np.ndarray | None = None  # kinematic trees: [L] int32 parent within the tree

    @property
    def n_chains(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_links_total(self) -> int:
        return int(self.offsets[-1])

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def chain(self, k: int) -> "ChainModel":
        a, b = int(self.offsets[k]), int(self.offsets[k + 1])
        return ChainModel(self.axes[a:b].copy(), self.frames[a:b].copy(),
                          self.inertias[a:b].copy(),
                          np.array([0, b - a], dtype=np.int64), self.gravity.copy(),
                          None if self.parents is None else self.parents[a:b].copy())


@dataclass
class States:
    q: np.ndarray
    qdot: np.ndarray
    tau: np.ndarray


def _unit(x: np.ndarray) -> np.ndarray:
    return x / np.linalg.norm(x, axis=-1, keepdims=True)


def _quat_to_rot(qu: np.ndarray) -> np.ndarray:
    w, x, y, z = qu[..., 0], qu[..., 1], qu[..., 2], qu[..., 3]
    R = np.empty(qu.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _skew(c: np.ndarray) -> np.ndarray:
    S = np.zeros(c.shape[:-1] + (3, 3))
    S[..., 0, 1], S[..., 0, 2] = -c[..., 2], c[..., 1]
    S[..., 1, 0], S[..., 1, 2] = c[..., 2], -c[..., 0]
    S[..., 2, 0], S[..., 2, 1] = -c[..., 1], c[..., 0]
    return S


def rigid_body_inertia(mass: np.ndarray, com: np.ndarray, I_c: np.ndarray) -> np.ndarray:
    """6x6 spatial inertia at the frame origin from mass, centre of mass and the
    rotational inertia about the centre of mass (all in the link frame).
    Returns [..., 6, 6]."""
    m = mass[..., None, None]
    C = _skew(com)
    J = np.zeros(mass.shape + (6, 6))
    J[..., :3, :3] = I_c - m * (C @ C)
    J[..., :3, 3:] = m * C
    J[..., 3:, :3] = -m * C
    J[..., 3:, 3:] = m * np.eye(3)
    return J


def offsets_from_lengths(lengths) -> np.ndarray:
    lengths = np.asarray(lengths, dtype=np.int64)
    off = np.zeros(lengths.shape[0] + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


def log_uniform_lengths(n_chains: int, lo: int, hi: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    n = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_chains)))
    return np.clip(n, lo, hi).astype(np.int64)


def random_chains(lengths, seed: int = 0, random_home_rotation: bool = False,
                  gravity=GRAVITY) -> ChainModel:
    """Draw ``len(lengths)`` independent serial chains of revolute joints."""
    if np.isscalar(lengths):
        lengths = [int(lengths)]
    off = offsets_from_lengths(lengths)
    L = int(off[-1])
    rng = np.random.default_rng(seed)
    axes = _unit(rng.standard_normal((L, 3)))
    lens = rng.uniform(0.1, 0.5, size=L)
    dirs = _unit(rng.standard_normal((L, 3)))
    masses = rng.uniform(0.5, 5.0, size=L)
    coms = rng.uniform(-0.05, 0.05, size=(L, 3))
    moments = rng.uniform(0.01, 0.1, size=(L, 3))
    Rp = _quat_to_rot(_unit(rng.standard_normal((L, 4))))
    if random_home_rotation:
        Rh = _quat_to_rot(_unit(rng.standard_normal((L, 4))))
    else:
        Rh = np.broadcast_to(np.eye(3), (L, 3, 3))
    I_c = Rp @ (moments[:, :, None] * np.swapaxes(Rp, -1, -2))
    J = rigid_body_inertia(masses, coms, I_c)
    frames = np.empty((L, 12))
    frames[:, :9] = Rh.reshape(L, 9)
    frames[:, 9:] = lens[:, None] * dirs
    return ChainModel(axes=np.ascontiguousarray(axes), frames=frames,
                      inertias=np.ascontiguousarray(J.reshape(L, 36)),
                      offsets=off, gravity=np.asarray(gravity, dtype=np.float64).copy())


def random_parents(lengths, seed: int = 0, p_branch: float = 0.3, p_base: float = 0.05):
    """Parent arrays of kinematic trees with the given link counts (links
    numbered parents first): link 0 sits on the base; link i > 0 continues the
    branch of link i-1, or with probability ``p_branch`` branches off a uniformly
    drawn earlier link, or with probability ``p_base`` starts a new branch on the
    base. One uniform draw per link, in link order, from its own stream."""
    if np.isscalar(lengths):
        lengths = [int(lengths)]
    rng = np.random.default_rng(seed)
    out = []
    for n in lengths:
        n = int(n)
        u = rng.uniform(size=max(n, 1))
        v = rng.uniform(size=max(n, 1))
        par = np.empty(n, dtype=np.int32)
        for i in range(n):
            if i == 0 or u[i] < p_base:
                par[i] = -1
            elif u[i] < p_base + p_branch:
                par[i] = int(v[i] * i)  # an earlier link, uniformly
            else:
                par[i] = i - 1
        out.append(par)
    return np.concatenate(out) if out else np.zeros(0, dtype=np.int32)


def random_trees(lengths, seed: int = 0, random_home_rotation: bool = False,
                 gravity=GRAVITY, p_branch: float = 0.3, p_base: float = 0.05) -> ChainModel:
    """Kinematic trees: the links of :func:`random_chains` (same draws, same
    seed) joined by :func:`random_parents` (seed + 1)."""
    m = random_chains(lengths, seed=seed, random_home_rotation=random_home_rotation,
                      gravity=gravity)
    m.parents = random_parents(m.lengths(), seed=seed + 1, p_branch=p_branch, p_base=p_base)
    return m


def random_loops(model: ChainModel, per_tree: int = 1, seed: int = 0, min_joints: int = 6):
    """Revolute loop joints closing each tree of ``model`` (``per_tree`` each):
    link b uniform over the tree's links, link a uniform over the tree's links
    and the base (-1), redrawn until the two paths to the base differ by at
    least ``min_joints`` joints, five of them in no other loop of the tree (so
    the loops' constraints are independent);
    the joint frames on either side are a rotation from a normalised normal
    quaternion and an offset U[-0.1, 0.1]^3 m. Returns a dict of arrays: tree,
    a, b (int32, link indices within the tree), frame_a, frame_b (K x 12, R
    row-major then p, in link a's (the base's) and link b's frames)."""
    rng = np.random.default_rng(seed)
    par = model.parents
    tree, A, B, FA, FB = [], [], [], [], []
    for t in range(model.n_chains):
        o, z = int(model.offsets[t]), int(model.offsets[t + 1])
        n = z - o

        def path(i):
            out = set()
            while i >= 0:
                out.add(i)
                i = int(par[o + i]) if par is not None else i - 1
            return out
        used = set()
        for _ in range(per_tree):
            for _try in range(1000):
                b = int(rng.integers(0, n))
                a = int(rng.integers(-1, n))
                joints = path(a) ^ path(b)
                if a != b and len(joints) >= min_joints and len(joints - used) >= 5:
                    used |= joints
                    break
            else:
                raise ValueError(f"tree {t} has no pair of links {min_joints} joints apart")
            fr = []
            for _side in range(2):
                R = _quat_to_rot(_unit(rng.standard_normal(4)))
                fr.append(np.concatenate([R.reshape(9), rng.uniform(-0.1, 0.1, size=3)]))
            tree.append(t); A.append(a); B.append(b); FA.append(fr[0]); FB.append(fr[1])
    return {"tree": np.array(tree, dtype=np.int32), "a": np.array(A, dtype=np.int32),
            "b": np.array(B, dtype=np.int32), "frame_a": np.array(FA).reshape(-1, 12),
            "frame_b": np.array(FB).reshape(-1, 12)}


def random_states(n_links_total: int, seed: int = 0, qdot_std: float = 1.0,
                  tau_std: float = 10.0) -> States:
    rng = np.random.default_rng(seed)
    q = rng.uniform(-np.pi, np.pi, size=n_links_total)
    qd = rng.standard_normal(n_links_total) * qdot_std
    tau = rng.standard_normal(n_links_total) * tau_std
    return States(q, qd, tau)


def replicate_model(model: ChainModel, n_problems: int):
    """Problem -> chain map for a batch of ``n_problems`` states all using chain 0
    of ``model`` (the shared-model batch), plus the packed state offsets."""
    n = int(model.offsets[1] - model.offsets[0])
    chain_index = np.zeros(n_problems, dtype=np.int32)
    state_offsets = np.arange(n_problems + 1, dtype=np.int64) * n
    return chain_index, state_offsets
