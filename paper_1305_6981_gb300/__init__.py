"""GB300 (sm_103a) FCIQMC walker cycle behind a C ABI (include/fciqmc.h)."""
from .fciqmc import Batch, Fciqmc, Partitioned, owners, rng_throughput, words_for  # noqa: F401
from .energy import EnergyFunctional, rdm_energy  # noqa: F401
