"""GB300-native pooled-chain pCN sampler for Bayesian quantum state tomography (arXiv:2501.17334).

``qst`` is the binding of the C ABI in ``include/qst.h`` (libqst.so, sm_103a);
``workload`` builds seeded synthetic Pauli-tomography problems; ``shard`` splits chains
over ranks and merges the pooled sums.
"""
__all__ = ["qst", "shard", "workload"]
