"""GB300 (sm_103a) implementation of the separable-density SOAP descriptor and the GAP
energy, forces and virial built on it (Caro, arXiv:1905.02142).

The compute path is the CUDA library in csrc/ behind the C ABI of include/soapgap.h;
``api`` is its Python binding.  Importing the package does not load the library; the
first ``SoapGap(...)`` does, and raises if the library has not been built.
"""


def __getattr__(name):
    if name in ("SoapGap", "SoapGapEnergy", "Structures", "SoapGapError"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
