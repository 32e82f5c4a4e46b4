"""CPU oracle (test infrastructure only): see ``oracle.gmres``."""
from . import gmres  # noqa: F401
