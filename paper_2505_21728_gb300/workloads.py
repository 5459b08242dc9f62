"""Named synthetic workloads shaped like the paper's transform settings.

Block sizes follow Sec. VI (4x4 and 8x8 secondary transforms, 35 intra
modes x 3 candidates = 105 sets); the 16x16 size extends the same
construction.  Residuals are Laplacian int16 values (the shape of
prediction residuals), drawn by ``inputs`` with fixed seeds.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import inputs


@dataclass
class Workload:
    name: str
    log2n: int
    rounds: int
    num_sets: int
    nblocks: int
    scale: float
    clip: tuple
    seed: int = 0
    skip_frac: float = 0.0
    description: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return 1 << self.log2n

    def params(self):
        q = inputs.angle_indices(self.num_sets, self.rounds, self.log2n, seed=self.seed)
        perms = inputs.permutations(self.num_sets, self.rounds, self.N, seed=self.seed)
        return q, perms

    def blocks(self, first: int = 0, count: int | None = None) -> np.ndarray:
        return inputs.laplacian_blocks(self.nblocks, self.N, self.scale, self.clip[0],
                                       self.clip[1], seed=self.seed, first_block=first,
                                       count=count)

    def set_indices(self) -> np.ndarray | None:
        if self.num_sets == 1 and self.skip_frac == 0:
            return np.zeros(self.nblocks, np.uint16)
        return inputs.set_indices(self.nblocks, self.num_sets, seed=self.seed,
                                  skip_frac=self.skip_frac)

    def generate(self) -> dict:
        q, perms = self.params()
        return {"angle_idx": q, "perms": perms, "x": self.blocks(), "sets": self.set_indices()}

    def bytes_fwd_inv(self) -> int:
        """Algorithmic HBM bytes of one forward + inverse: int16 in and int32
        out, then int32 in and int16 out, plus the 2-byte set index read in
        each direction."""
        return self.nblocks * (2 * self.N + 4 * self.N + 2) * 2


_REGISTRY = {
    "hygt4x4_r2": Workload(
        "hygt4x4_r2", log2n=4, rounds=2, num_sets=1, nblocks=65536, scale=12.0,
        clip=(-512, 511), seed=0,
        description="4x4 non-separable HyGT (N=16), 2 rounds, one set, 65,536 Laplace(12) "
                    "int16 blocks clipped to [-512, 511]"),
    "hygt8x8_r2_s105": Workload(
        "hygt8x8_r2_s105", log2n=6, rounds=2, num_sets=105, nblocks=4194304, scale=8.0,
        clip=(-1024, 1023), seed=0,
        description="8x8 non-separable HyGT (N=64), 2 rounds, 105 sets (35 modes x 3), "
                    "4,194,304 Laplace(8) int16 blocks clipped to [-1024, 1023], set index "
                    "uniform over 0..104"),
    "hygt16x16_r3_s16": Workload(
        "hygt16x16_r3_s16", log2n=8, rounds=3, num_sets=16, nblocks=16777216, scale=4.0,
        clip=(-2048, 2047), seed=0,
        description="16x16 non-separable HyGT (N=256), 3 rounds, 16 sets, 16,777,216 "
                    "Laplace(4) int16 blocks clipped to [-2048, 2047]"),
}


@dataclass
class MixedWorkload:
    """A frame sequence tiled into 4x4, 8x8 and 16x16 blocks (one class per
    block size, each with its own transform sets)."""
    name: str
    frames: int
    width: int
    height: int
    num_sets: int
    scale: float
    clip: tuple
    skip_frac: float
    rounds: tuple = (2, 2, 3)       # rounds for N = 16, 64, 256
    area_mix: tuple = (0.50, 0.35, 0.15)
    seed: int = 0
    description: str = ""
    scale_down: int = 1             # divide the block counts (small test cases)

    def counts(self):
        t = inputs.mixed_frame_tiling(self.frames, self.width, self.height, self.seed,
                                      self.area_mix)["blocks"]
        return tuple(max(1, c // self.scale_down) for c in t)

    def classes(self):
        """One Workload per block size (N = 16, 64, 256)."""
        out = []
        for k, (log2n, nb) in enumerate(zip((4, 6, 8), self.counts())):
            out.append(Workload("%s/N%d" % (self.name, 1 << log2n), log2n=log2n,
                                rounds=self.rounds[k], num_sets=self.num_sets, nblocks=nb,
                                scale=self.scale, clip=self.clip, seed=self.seed + 17 * (k + 1),
                                skip_frac=self.skip_frac))
        return out

    @property
    def nblocks(self):
        return sum(self.counts())

    def bytes_fwd_inv(self):
        return sum(c.bytes_fwd_inv() for c in self.classes())


_MIXED = {
    "mixed_frame_2160p16": MixedWorkload(
        "mixed_frame_2160p16", frames=16, width=3840, height=2160, num_sets=105, scale=6.0,
        clip=(-512, 511), skip_frac=0.10,
        description="16 frames of 3840x2160 residual tiled into 4x4 / 8x8 / 16x16 blocks "
                    "(50/35/15% of the area, seeded), set index uniform over 0..104, 10% of "
                    "blocks without a transform, Laplace(6) int16 clipped to [-512, 511]; "
                    "N=16 and N=64 with 2 rounds, N=256 with 3 rounds"),
}


@dataclass
class FitWorkload:
    """Differentiable FP32 HyGT on correlated patches (angle fitting)."""
    name: str
    log2n: int
    rounds: int
    nvec: int
    keep: int                       # K: coefficients whose energy is kept
    seed: int = 0
    description: str = ""

    @property
    def N(self) -> int:
        return 1 << self.log2n

    def patches(self, count=None) -> np.ndarray:
        side = int(round(self.N ** 0.5))
        return inputs.ar1_patches(self.nvec if count is None else count, side, seed=self.seed)

    def theta0(self) -> np.ndarray:
        return inputs.theta_uniform((1, self.rounds, self.log2n, self.N // 2), seed=self.seed)


_FIT = {
    "hygt8x8_r4_fit": FitWorkload(
        "hygt8x8_r4_fit", log2n=6, rounds=4, nvec=1048576, keep=8, seed=0,
        description="differentiable FP32 HyGT, N=64, 4 rounds (768 angles), 1,048,576 8x8 "
                    "patches: half separable AR(1) (0.95, 0.9), half 45-degree rotated AR(1) "
                    "(0.97 / 0.6); loss = energy outside the first 8 coefficients"),
}


def get_fit(name: str) -> FitWorkload:
    return _FIT[name]


def get_mixed(name: str, scale_down: int = 1) -> MixedWorkload:
    import dataclasses
    w = _MIXED[name]
    return dataclasses.replace(w, scale_down=scale_down) if scale_down != 1 else w


def truncated(w: Workload, nblocks: int) -> Workload:
    """The first nblocks blocks of a workload (same parameters and seeds)."""
    import dataclasses
    n = min(int(nblocks), w.nblocks)
    return dataclasses.replace(w, name="%s[:%d]" % (w.name, n), nblocks=n)


def get(name: str) -> Workload:
    """A named workload, or one block-size class of a mixed batch
    ("mixed_frame_2160p16/N16", "/N64", "/N256")."""
    if name in _REGISTRY:
        return _REGISTRY[name]
    base, _, cls = name.partition("/")
    if base in _MIXED and cls:
        for c in _MIXED[base].classes():
            if c.name == name:
                return c
    raise KeyError(name)


def names():
    return sorted(_REGISTRY)
