"""GB300 (sm_103a) FCIQMC walker cycle behind a C ABI (include/fciqmc.h)."""
from .fciqmc import Fciqmc, words_for  # noqa: F401
