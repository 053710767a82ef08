"""GB300-native aperture-aware proton Monte Carlo dose engine.

The compute path is the C-ABI library built from csrc/ (see include/vpmc.h);
`paper_2307_01416_gb300.vpmc` is its Python binding and
`paper_2307_01416_gb300.workloads` holds the seeded synthetic inputs.
"""
__all__ = ["vpmc", "workloads"]
