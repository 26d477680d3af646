"""The five workload configurations as data (inputs, model shape, parameter draw).

Each stands in for a class of the paper's periodic metallic workloads (Section IV) with the
shapes and sizes of the benchmark configurations:
  C1  fcc unary 108 atoms, level 8 (small case, every atom checkable)
  C2  B2 binary 40^3 bcc cells (128,000 atoms), level 16
  C3  512 training configurations of 8-256 atoms, level-16 ternary student
  C4  fcc ternary random solid solution 64^3 cells (1,048,576 atoms), level 20 (benchmark)
  C5  liquid-like quaternary, 2,097,152 atoms, R_cut 6 A, level 24
`workload(name).inputs(seed)` returns the batch dict (see synth.py; seed None = the workload's
own structure seed), `.desc()` the model descriptor and `.theta()` the seeded parameter vector.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable

from . import synth


@dataclass(frozen=True)
class Workload:
    name: str
    n_types: int
    lev_max: int
    r_cut: float
    theta_seed: int
    nbar: float                      # mean neighbor count for the parameter scale (reading R14)
    input_seed: int
    make_inputs: Callable[[int], dict] = field(repr=False)
    r_min: float = 2.0
    n_q: int = 8

    def inputs(self, seed: int | None = None) -> dict:
        return self.make_inputs(self.input_seed if seed is None else seed)

    def desc(self):
        from . import api
        return api.make_desc(self.n_types, self.lev_max, self.n_q, self.r_min, self.r_cut)

    def theta(self):
        from . import api
        d = self.desc()
        basis = api.mtp_describe_basis(d)
        sizes = api.mtp_describe(d)
        nu_sum = [sum(nu for _, nu in labs) for labs, _ in basis]
        nf = [len(labs) for labs, _ in basis]
        return synth.draw_theta(self.theta_seed, self.n_types, sizes["n_rad"], self.n_q, nu_sum, nf, self.r_min,
                                self.r_cut, self.nbar)


WORKLOADS = {
    "C1": Workload("fcc unary 108 atoms", 1, 8, 5.0, 11, 42.0, 1, lambda s: synth.fcc_unary_108(seed=s)),
    "C2": Workload("B2 binary 40^3 cells", 2, 16, 5.0, 22, 58.0, 2, lambda s: synth.b2_binary(seed=s, n=40)),
    "C3": Workload("512 training configurations", 3, 16, 5.0, 34, 42.0, 3, lambda s: synth.training_batch(seed=s)),
    "C4": Workload("fcc ternary 64^3 cells", 3, 20, 5.0, 44, 42.0, 4, lambda s: synth.fcc_ternary(seed=s, n=64)),
    "C5": Workload("liquid quaternary 2,097,152 atoms", 4, 24, 6.0, 55, 76.0, 5,
                   lambda s: synth.liquid_rsa(seed=s, tiles=4)),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]
