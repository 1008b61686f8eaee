"""GB300-native residual-specific partial-jet PINN kernels (sm_103a).

Importing the package loads nothing native; ``paper_2606_29702_gb300.jet``
loads the CUDA library ``libjet`` and fails loudly if it is missing.
"""
