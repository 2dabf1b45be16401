"""Oracle package -- test infrastructure only (see reference.py)."""
from .reference import *  # noqa: F401,F403
from .reference import TECTONIC, TW  # noqa: F401
